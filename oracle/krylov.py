"""Right-preconditioned flexible GMRES (Saad 1993, the outer Krylov method of Sec. 3.3 and Sec. 5).

FGMRES(m) from x_0 = 0: Arnoldi on w = L z_j with z_j = M(v_j) stored (the preconditioner may
change between iterations), orthogonalisation by classical Gram-Schmidt applied twice (CGS2),
Givens rotations on the Hessenberg matrix, stop when the rotated residual estimate falls to
rtol * ||b||_2 or after max_it iterations; at the end of each cycle x += Z_j y with
y = H_j^{-1} g_j.  The returned x is gauge-fixed (null-space components removed).

Pinned by: for M = I the residual after k steps equals the minimum of ||b - L y|| over the
Krylov space K_k(L, b) computed by brute-force least squares; the residual estimate equals the
true residual; exact termination in n steps on an n-dimensional problem.
"""
import numpy as np


def fgmres(apply_L, apply_M, b, rtol=1e-8, max_it=100, restart=100, project=None):
    n = b.size
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    hist = [bnorm]
    its = 0
    converged = bnorm == 0.0
    while not converged and its < max_it:
        r = b - apply_L(x) if its > 0 else b.copy()
        beta = np.linalg.norm(r)
        m = min(restart, max_it - its)
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = apply_M(V[j])
            w = apply_L(Z[j])
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            h = h + h2
            hn = np.linalg.norm(w)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            if hn > 0:
                V[j + 1] = w / hn
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / d
            sn[j] = H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= rtol * bnorm or hn == 0.0:
                converged = True
                break
            if its >= max_it:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
    if project is not None:
        x = project(x)
    return x, its, np.array(hist), converged

"""Smoothers on one multigrid level (Sec. 3.3).

Additive Vanka (Alg. 2, restricted additive Schwarz, taken with one-cell subdomains as the
per-cell additive Vanka form): the residual is formed once from the incoming iterate; for every
cell c the 5x5 saddle-point patch operator L_c = R_c L R_c^T on the dofs
(u_{i-1/2,j}, u_{i+1/2,j}, v_{i,j-1/2}, v_{i,j+1/2}, p_{i,j}) is solved against R_c r, and the
corrections are weighted (1/2 on the four faces, each shared by two cells, 1 on the pressure)
and summed.  One sweep is x <- x + omega * sum_c W_c R_c^T L_c^{-1} R_c (b - L x).

Schur-complement smoother (Eqs. fact-Stokes-IB and approx-fact-Stokes-IB):
    y  = At^{-1} r_u,   dp = Mt^{-1}(r_p + D y),   du = y - At^{-1}(G dp),   x <- x + omega (du, dp)
At^{-1}: a fixed number of Chebyshev iterations on A_IB with point (Jacobi) preconditioning;
Mt^{-1}: a fixed number of Chebyshev iterations on D At^{-1} G preconditioned by the diagonal of
the sparse approximate Schur complement Mh = D diag(A_IB)^{-1} G.  The paper relaxes with
Gauss-Seidel; here the diagonal (Jacobi) point relaxation is used instead, so that every level is
one parallel pass.

Chebyshev acceleration follows the textbook recurrence (Saad, Iterative Methods for Sparse
Linear Systems, Algorithm 12.1) with x_0 = 0 on the interval [lo, hi] * lambda_max, where
lambda_max of the Jacobi-preconditioned operator is estimated by a fixed number of power
iterations from the deterministic start vector of ``hash_vector``.

Pinned by: Vanka leaves the exact solution fixed and its action equals a brute-force sum of
patch solves with independently derived dof lists; Chebyshev's residual equals the closed-form
polynomial T_k((theta - t)/delta) / T_k(theta/delta) on diagonal operators; the SC formula with
exact inner inverses reproduces L^{-1}.
"""
import numpy as np

from .mac import cell_index

VANKA_WEIGHTS = np.array([0.5, 0.5, 0.5, 0.5, 1.0])


def vanka_patch_dofs(N):
    """(N^2, 5) global dof indices of every cell's patch, cells row-major [j][i]."""
    n = N * N
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    i, j = i.ravel(), j.ravel()
    return np.stack([cell_index(N, i, j), cell_index(N, i + 1, j),
                     n + cell_index(N, i, j), n + cell_index(N, i, j + 1),
                     2 * n + cell_index(N, i, j)], axis=1)


def vanka_patches(L, dofs):
    """L_c = R_c L R_c^T for every cell, (ncell, 5, 5)."""
    rows = np.repeat(dofs[:, :, None], 5, axis=2)
    cols = np.repeat(dofs[:, None, :], 5, axis=1)
    vals = np.asarray(L[rows.ravel(), cols.ravel()]).reshape(dofs.shape[0], 5, 5)
    return vals


def vanka_sweep(L, dofs, patches, x, b, omega):
    r = b - L @ x
    delta = np.linalg.solve(patches, r[dofs][..., None])[..., 0]
    dx = np.zeros_like(x)
    np.add.at(dx, dofs.ravel(), (delta * VANKA_WEIGHTS).ravel())
    return x + omega * dx


def hash_vector(n):
    """Deterministic start vector: Knuth's multiplicative hash of (k+1), mapped to [-1/2, 1/2)."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    return ((k * np.uint64(2654435761)) % np.uint64(2 ** 32)).astype(np.float64) / 2.0 ** 32 - 0.5


def power_max(apply_op, dinv, n, iters):
    """Estimate of the largest eigenvalue of diag^{-1} Op: ||w|| after `iters` normalised steps."""
    v = hash_vector(n)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = dinv * apply_op(v)
        lam = np.linalg.norm(w)
        v = w / lam
    return lam


def chebyshev(apply_op, dinv, b, lam_max, iters, lo=0.1, hi=1.1):
    """`iters` Chebyshev iterations for Op x = b from x_0 = 0, preconditioner diag^{-1}."""
    lmin, lmax = lo * lam_max, hi * lam_max
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b.copy()
    d = (dinv * r) / theta
    x = np.zeros_like(b)
    for k in range(iters):
        x = x + d
        if k == iters - 1:
            break
        r = r - apply_op(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
    return x


def sc_apply(r, nu, Ainv, Minv, G, D):
    """Approximate block-factorised inverse applied to r = (r_u, r_p)."""
    y = Ainv(r[:nu])
    dp = Minv(r[nu:] + D @ y)
    du = y - Ainv(G @ dp)
    return np.concatenate([du, dp])


def sc_sweep(L, G, D, AIB, dA, dM, lamA, lamM, x, b, omega, cheb_iters, lo=0.1, hi=1.1):
    nu = G.shape[0]
    dAinv = 1.0 / dA
    dMinv = 1.0 / dM

    def Ainv(q):
        return chebyshev(lambda z: AIB @ z, dAinv, q, lamA, cheb_iters, lo, hi)

    def Mop(q):
        return D @ Ainv(G @ q)

    def Minv(q):
        return chebyshev(Mop, dMinv, q, lamM, cheb_iters, lo, hi)

    r = b - L @ x
    return x + omega * sc_apply(r, nu, Ainv, Minv, G, D)


def fgmres_smooth(L, B, x, b, k):
    """The paper's smoothing step (Sec. 3.3): k iterations of flexible GMRES on the residual
    equation L e = b - L x, preconditioned by the basic smoother B (B(v): one undamped sweep on
    right-hand side v from a zero guess), then x + e.  Classical Gram-Schmidt applied twice; the
    iterations stop early when the new Arnoldi vector vanishes.  k = the number of sweeps the
    damped form would take, so both apply B the same number of times."""
    r = b - L @ x
    beta = np.linalg.norm(r)
    if beta == 0.0:
        return x.copy()
    n = r.size
    V = np.zeros((n, k + 1))
    Z = np.zeros((n, k))
    H = np.zeros((k + 1, k))
    V[:, 0] = r / beta
    m = 0
    for j in range(k):
        Z[:, j] = B(V[:, j])
        w = L @ Z[:, j]
        h = V[:, :j + 1].T @ w
        w = w - V[:, :j + 1] @ h
        h2 = V[:, :j + 1].T @ w
        w = w - V[:, :j + 1] @ h2
        H[:j + 1, j] = h + h2
        H[j + 1, j] = np.linalg.norm(w)
        m = j + 1
        if H[j + 1, j] == 0.0:
            break
        V[:, j + 1] = w / H[j + 1, j]
    rhs = np.zeros(m + 1)
    rhs[0] = beta
    y = np.linalg.lstsq(H[:m + 1, :m], rhs, rcond=None)[0]
    return x + Z[:, :m] @ y

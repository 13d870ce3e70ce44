"""The semi-implicit Stokes-IB linear system and three independent exact solves of it
(Sec. 2.2, Eqs. system-impib and matrix-impib).

Eliminated system (Eq. matrix-impib):
    L_IB = [[A - dt S K J, G], [-D, 0]],   right-hand side (g + S K X^n, 0).
With S = J^T/h^2, K symmetric and -D = G^T, L_IB is symmetric (indefinite).

Periodic-domain reading (the paper's tests use Dirichlet cavity walls; the problems here are
periodic).  The kernel of L_IB is spanned by the constant pressure and, when rho = 0, by the two
constant velocity components (J maps constants to constants and K annihilates translations).
The right-hand side is made consistent by removing the mean of each velocity component when
rho = 0 (S K X^n has zero mean exactly), and every solution is gauge-fixed to zero mean in the
null-space components.  ``project`` is that gauge step.

Exact solves, each independent of the others:
  solve_direct       -- sparse LU of L_IB bordered by the null-space constraints
  solve_full_system  -- sparse LU of the 3x3 (u, p, X^{n+1}) system of Eq. system-impib
  solve_lagrangian   -- Lagrangian elimination (the Mori-Peskin / Ceniceros et al. approach the
                        paper cites): a dense (2M x 2M) solve for X^{n+1} built on an FFT solve
                        of periodic MAC Stokes with the exact Fourier symbols (fft_stokes).
Pinned by: agreement of the three, symmetry, discrete incompressibility, and fft_stokes against
the sparse operator on Fourier modes.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import ib, mac


def stokes_ib_operator(N, rho, mu, dt, X, edges, kappa):
    A = mac.momentum(N, rho, mu, dt)
    B = ib.ib_operator(N, X, edges, kappa)
    G = mac.gradient(N)
    D = mac.divergence(N)
    return sp.bmat([[A - dt * B, G], [-D, None]], format="csr")


def operator_of(prob):
    s = prob.structure
    return stokes_ib_operator(prob.N, prob.rho, prob.mu, prob.dt, s.X, s.edges, s.kappa)


def null_basis(N, rho):
    """Orthonormal basis (3N^2 x k) of the kernel of L_IB on the periodic grid."""
    n = N * N
    cols = []
    blocks = (0, 1, 2) if rho == 0.0 else (2,)
    for b in blocks:
        z = np.zeros(3 * n)
        z[b * n:(b + 1) * n] = 1.0 / N
        cols.append(z)
    return np.stack(cols, axis=1)


def project(w, N, rho):
    """Remove the null-space components (the gauge step): zero mean per block in the kernel."""
    n = N * N
    w = np.array(w, dtype=np.float64, copy=True)
    blocks = (0, 1, 2) if rho == 0.0 else (2,)
    for b in blocks:
        w[b * n:(b + 1) * n] -= w[b * n:(b + 1) * n].mean()
    return w


def rhs(prob, add_SKXn=True):
    """b = (g + S K X^n, 0) with the velocity means removed when rho = 0."""
    N = prob.N
    n = N * N
    s = prob.structure
    b = np.zeros(3 * n)
    b[:2 * n] = prob.g[:2 * n]
    if add_SKXn and s.M > 0:
        F = ib.stiffness(s.M, s.edges, s.kappa) @ s.X
        b[:2 * n] += ib.spread_force(N, s.X, F)
    if prob.rho == 0.0:
        for c in (0, 1):
            b[c * n:(c + 1) * n] -= b[c * n:(c + 1) * n].mean()
    return b


def solve_direct(L, b, N, rho):
    """Solve L w = b with Z^T w = 0 through the bordered matrix [[L, Z], [Z^T, 0]] (sparse LU)."""
    Z = null_basis(N, rho)
    k = Z.shape[1]
    Zs = sp.csr_matrix(Z)
    Bm = sp.bmat([[L, Zs], [Zs.T, None]], format="csc")
    sol = spla.splu(Bm).solve(np.concatenate([b, np.zeros(k)]))
    return sol[:-k], sol[-k:]


def solve_full_system(prob, add_SKXn=True):
    """Solve the (u, p, X^{n+1}) system of Eq. system-impib directly; returns (w, X^{n+1}).

    Rows: A u + G p - S K X = g;  -D u = 0;  -J u + X/dt = X^n/dt (per component).
    Gauge rows fix zero mean of p and, for rho = 0, of u and v.  With add_SKXn=False the
    spring force acts on the displacement X^{n+1}-X^n only (the homogeneous form).
    """
    N, n = prob.N, prob.N * prob.N
    s = prob.structure
    M = s.M
    A = mac.momentum(N, prob.rho, prob.mu, prob.dt)
    G = mac.gradient(N)
    D = mac.divergence(N)
    K = ib.stiffness(M, s.edges, s.kappa)
    Ss = [ib.spread_matrix(N, s.X, c) for c in (0, 1)]
    Js = [ib.interp_matrix(N, s.X, c) for c in (0, 1)]
    SK = sp.block_diag([Ss[0] @ K, Ss[1] @ K])                   # (2n x 2M), X ordered [x | y]
    Jb = sp.block_diag(Js)                                       # (2M x 2n)
    I2M = sp.identity(2 * M) / prob.dt
    Z = sp.csr_matrix(null_basis(N, prob.rho))
    k = Z.shape[1]
    Zpad = sp.vstack([Z, sp.csr_matrix((2 * M, k))])
    top = sp.bmat([[A, G, -SK], [-D, None, None], [-Jb, None, I2M]], format="csr")
    Bm = sp.bmat([[top, Zpad], [Zpad.T, None]], format="csc")
    g = np.zeros(2 * n)
    g[:] = prob.g[:2 * n]
    if prob.rho == 0.0:
        for c in (0, 1):
            g[c * n:(c + 1) * n] -= g[c * n:(c + 1) * n].mean()
    Xn = np.concatenate([s.X[:, 0], s.X[:, 1]])
    rhs_x = Xn / prob.dt
    if not add_SKXn:
        # homogeneous form: unknown is the displacement, force K(X^{n+1} - X^n)
        rhs_x = np.zeros(2 * M)
    r = np.concatenate([g, np.zeros(n), rhs_x, np.zeros(k)])
    sol = spla.splu(Bm).solve(r)
    w = sol[:3 * n]
    Xnew = sol[3 * n:3 * n + 2 * M]
    if not add_SKXn:
        Xnew = Xnew + Xn
    return w, np.stack([Xnew[:M], Xnew[M:]], axis=1)


def fft_stokes(N, rho, mu, dt, f):
    """Solve [[A, G], [-D, 0]] w = f on the periodic MAC grid with the exact Fourier symbols.

    With F_k = sum_n f_n exp(-2 pi i k n / N) a shift q_{i-1} has symbol exp(-i theta):
      Lap -> -(4 sin^2(theta_1/2) + 4 sin^2(theta_2/2)) / h^2
      G   -> ((1 - exp(-i theta_1))/h, (1 - exp(-i theta_2))/h),  D -> ((exp(i theta_1) - 1)/h, ...)
    Each mode is a 3x3 complex system; the zero mode keeps p = 0 and u = f/(rho/dt) (0 if rho = 0).
    """
    h = 1.0 / N
    n = N * N
    fu = np.fft.fft2(f[:n].reshape(N, N))
    fv = np.fft.fft2(f[n:2 * n].reshape(N, N))
    fp = np.fft.fft2(f[2 * n:].reshape(N, N))
    k = np.arange(N)
    th2, th1 = np.meshgrid(2 * np.pi * k / N, 2 * np.pi * k / N, indexing="ij")  # [j][i]
    lam = -(4 * np.sin(th1 / 2) ** 2 + 4 * np.sin(th2 / 2) ** 2) / h ** 2
    a = rho / dt - mu * lam
    g1 = (1 - np.exp(-1j * th1)) / h
    g2 = (1 - np.exp(-1j * th2)) / h
    d1 = (np.exp(1j * th1) - 1) / h
    d2 = (np.exp(1j * th2) - 1) / h
    Mx = np.zeros((N, N, 3, 3), dtype=complex)
    Mx[..., 0, 0] = a
    Mx[..., 0, 2] = g1
    Mx[..., 1, 1] = a
    Mx[..., 1, 2] = g2
    Mx[..., 2, 0] = -d1
    Mx[..., 2, 1] = -d2
    rhs_ = np.stack([fu, fv, fp], axis=-1)
    # the zero mode is singular in p (and in u, v when rho = 0): replace by the gauge rows
    Mx[0, 0] = np.eye(3) * (a[0, 0] if a[0, 0] != 0 else 1.0)
    Mx[0, 0, 2, 2] = 1.0
    rhs_[0, 0, 2] = 0.0
    if a[0, 0] == 0:
        rhs_[0, 0, 0] = 0.0
        rhs_[0, 0, 1] = 0.0
    sol = np.linalg.solve(Mx, rhs_[..., None])[..., 0]
    out = np.concatenate([np.real(np.fft.ifft2(sol[..., c])).ravel() for c in range(3)])
    return out


def solve_lagrangian(prob, add_SKXn=True):
    """Lagrangian elimination: (I - dt J Sigma S K) X = X^n + dt J Sigma g, then w = Sigma(g + S K X).

    Sigma is fft_stokes (the periodic Stokes solution operator).  Returns (w, X^{n+1}).
    """
    N, n = prob.N, prob.N * prob.N
    s = prob.structure
    M = s.M
    K = ib.stiffness(M, s.edges, s.kappa).toarray()
    g = np.zeros(3 * n)
    g[:2 * n] = prob.g[:2 * n]
    if prob.rho == 0.0:
        for c in (0, 1):
            g[c * n:(c + 1) * n] -= g[c * n:(c + 1) * n].mean()

    def Sigma(f):
        return fft_stokes(N, prob.rho, prob.mu, prob.dt, f)

    def SK_of(Y):   # Y (M x 2) -> Eulerian force on faces (3n,)
        F = K @ Y
        out = np.zeros(3 * n)
        out[:2 * n] = ib.spread_force(N, s.X, F)
        return out

    # dense T = J Sigma S K on the 2M stacked unknowns [x | y]
    T = np.zeros((2 * M, 2 * M))
    for col in range(2 * M):
        Y = np.zeros((M, 2))
        Y[col % M, col // M] = 1.0
        U = ib.interp_velocity(N, s.X, Sigma(SK_of(Y)))
        T[:, col] = np.concatenate([U[:, 0], U[:, 1]])
    Xn = np.concatenate([s.X[:, 0], s.X[:, 1]])
    U0 = ib.interp_velocity(N, s.X, Sigma(g))
    if add_SKXn:
        rhs_ = Xn + prob.dt * np.concatenate([U0[:, 0], U0[:, 1]])
        Xv = np.linalg.solve(np.eye(2 * M) - prob.dt * T, rhs_)
        Xm = np.stack([Xv[:M], Xv[M:]], axis=1)
        w = Sigma(g + SK_of(Xm))
    else:
        rhs_ = prob.dt * np.concatenate([U0[:, 0], U0[:, 1]])
        Dv = np.linalg.solve(np.eye(2 * M) - prob.dt * T, rhs_)
        Dm = np.stack([Dv[:M], Dv[M:]], axis=1)
        w = Sigma(g + SK_of(Dm))
        Xm = s.X + Dm
    return w, Xm

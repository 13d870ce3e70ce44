"""The paper's lid-driven cavity (Sec. 5): the unit square with no-slip walls, and on the top wall
the regularised lid u(x, 1) = (1 - cos 2 pi x)/2, v = 0.  Test infrastructure: a plain FP64 CPU
restatement on the MAC grid with walls, used to check GPU results; it shares no code with the CUDA
path.

Readings (the paper treats its physical boundaries as in earlier work that it does not restate):
- The grid is the N x N MAC grid of the periodic layout, [u | v | p] with N^2 entries each,
  row-major [j][i].  The faces on its seam, u(0, j) at x = 0 (= 1) and v(i, 0) at y = 0 (= 1), lie
  on the walls: their normal velocity is a boundary value (0), not an unknown.  The unknowns are the
  other 3 N^2 - 2 N entries, in the layout's order (`interior`).
- Tangential velocity at a wall enters the five-point Laplacian through a ghost value extrapolated
  linearly across the wall: q_ghost = 2 q_wall - q_inside.  The lid's value is the only nonzero
  q_wall; it moves to the right-hand side (`lid_rhs`).
- G and D are the MAC differences with the wall faces removed, so D = -G^T; the kernel of the
  operator is the constant pressure (the velocity has Dirichlet conditions).
- Transfers: the RT0 velocity prolongation of the periodic grid, restricted to the unknowns (a
  coarse wall face carries 0); bilinear pressure prolongation with the coarse value reflected across
  a wall (the neighbour outside the domain is the cell itself); pressure restriction averages the
  four fine cells; R_u = P_u^T / 4.
- Vanka patches: the cell's faces that are unknowns and its pressure, weights 1/2 and 1.
- The structure must keep its Peskin support inside the domain (markers at least 2.5 h from the
  walls), so interpolation and spreading never meet a wall.

Pinned by (tests/test_oracle_cavity.py): D = -G^T and symmetry; the operator equals the periodic
operator on rows away from the walls; second-order convergence to manufactured divergence-free
Stokes solutions with no-slip walls, one of them driven by the lid (which fixes the lid's
right-hand side term); Cauchy convergence of the lid-driven flow; the RT0 identity
D_f P_u = Inj D_c; the pressure prolongation's linear reproduction and locality at the walls;
V-cycle and FGMRES convergence with an immersed structure.
"""
import numpy as np
import scipy.sparse as sp

from . import ib, smoothers, transfer
from .mac import cell_index


def interior(N):
    """Indices (into the 3 N^2 layout) of the unknowns: every entry but u(0, j) and v(i, 0)."""
    n = N * N
    mask = np.ones(3 * n, dtype=bool)
    j = np.arange(N)
    mask[cell_index(N, 0, j)] = False           # u on the x = 0 (= 1) wall
    mask[n + cell_index(N, j, 0)] = False       # v on the y = 0 (= 1) wall
    return np.flatnonzero(mask)


def embed(N, w):
    """Unknown vector -> 3 N^2 layout with zeros on the wall faces."""
    out = np.zeros(3 * N * N)
    out[interior(N)] = w
    return out


def _velocity_block(N, rho, mu, dt, comp):
    """(rho/dt) I - mu Lap for one velocity component on the 3N^2-layout indices of that component,
    with the wall rules; returns (rows, cols, vals) in component-local indices 0..N^2-1."""
    h = 1.0 / N
    c = mu / (h * h)
    rows, cols, vals = [], [], []
    for j in range(N):
        for i in range(N):
            if (comp == 0 and i == 0) or (comp == 1 and j == 0):
                continue                                      # wall face, not an unknown
            r = j * N + i
            diag = rho / dt + 4.0 * c
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ii, jj = i + di, j + dj
                normal = (di != 0) if comp == 0 else (dj != 0)
                if normal:
                    # along the component's own direction: a neighbour on the wall is a boundary
                    # value (0); index N wraps to the wall face 0
                    if (comp == 0 and ii % N == 0) or (comp == 1 and jj % N == 0):
                        continue
                    rows.append(r)
                    cols.append(cell_index(N, ii, jj))
                    vals.append(-c)
                else:
                    # across a tangential wall: ghost = 2 q_wall - q, i.e. +c on the diagonal (q_wall
                    # goes to the right-hand side)
                    if not (0 <= ii < N and 0 <= jj < N):
                        diag += c
                        continue
                    rows.append(r)
                    cols.append(jj * N + ii)
                    vals.append(-c)
            rows.append(r)
            cols.append(r)
            vals.append(diag)
    return np.array(rows), np.array(cols), np.array(vals)


def momentum(N, rho, mu, dt):
    """A = (rho/dt) I - mu Lap on the velocity unknowns (u block, then v block), sparse."""
    n = N * N
    blocks = []
    for comp in (0, 1):
        r, c_, v = _velocity_block(N, rho, mu, dt, comp)
        blocks.append(sp.csr_matrix((v, (r, c_)), shape=(n, n)))
    A = sp.block_diag(blocks, format="csr")
    vel = interior(N)[: 2 * n - 2 * N]
    return A[vel][:, vel].tocsr()


def gradient(N):
    """G: pressure -> velocity unknowns, (p(i,j) - p(i-1,j))/h on u(i,j), (p(i,j) - p(i,j-1))/h on v."""
    h = 1.0 / N
    n = N * N
    rows, cols, vals = [], [], []
    for j in range(N):
        for i in range(N):
            if i > 0:
                rows += [j * N + i, j * N + i]
                cols += [j * N + i, j * N + i - 1]
                vals += [1.0 / h, -1.0 / h]
            if j > 0:
                rows += [n + j * N + i, n + j * N + i]
                cols += [j * N + i, (j - 1) * N + i]
                vals += [1.0 / h, -1.0 / h]
    G = sp.csr_matrix((vals, (rows, cols)), shape=(2 * n, n))
    vel = interior(N)[: 2 * n - 2 * N]
    return G[vel].tocsr()


def divergence(N):
    """D u on the cells, (u(i+1,j) - u(i,j) + v(i,j+1) - v(i,j))/h, wall faces 0 (= -G^T)."""
    return (-gradient(N).T).tocsr()


def ib_operator(N, X, edges, kappa):
    """[S K J] on the velocity unknowns: the periodic operator restricted to them (the Peskin support
    of every marker stays inside the domain)."""
    h = 1.0 / N
    if X.shape[0] and (X.min() < 2.5 * h or X.max() > 1.0 - 2.5 * h):
        raise ValueError("markers must stay 2.5 h away from the walls")
    B = ib.ib_operator(N, X, edges, kappa)
    vel = interior(N)[: 2 * N * N - 2 * N]
    return B[vel][:, vel].tocsr()


def operator(N, rho, mu, dt, X, edges, kappa):
    """L = [[A - dt [SKJ], G], [-D, 0]] on the unknowns."""
    A = momentum(N, rho, mu, dt)
    B = ib_operator(N, X, edges, kappa)
    G = gradient(N)
    D = divergence(N)
    return sp.bmat([[A - dt * B, G], [-D, None]], format="csr")


def lid_velocity(x):
    return 0.5 * (1.0 - np.cos(2.0 * np.pi * x))


def lid_rhs(N, mu):
    """The lid's contribution to the momentum right-hand side: 2 mu u_lid(x_i) / h^2 on the top row of
    u faces (the ghost value's known part), zero elsewhere; on the unknowns."""
    h = 1.0 / N
    out = np.zeros(3 * N * N)
    i = np.arange(1, N)
    out[cell_index(N, i, N - 1)] = 2.0 * mu * lid_velocity(i * h) / (h * h)
    return out[interior(N)]


def null_basis(N):
    """Orthonormal basis of the kernel: the constant pressure."""
    nv = 2 * N * N - 2 * N
    z = np.zeros(nv + N * N)
    z[nv:] = 1.0 / N
    return z[:, None]


def project(w, N):
    """Remove the pressure mean."""
    nv = 2 * N * N - 2 * N
    out = w.copy()
    out[nv:] -= out[nv:].mean()
    return out


def solve_direct(L, b, N):
    """Gauge-fixed exact solve: (L + Z Z^T) w = b - Z Z^T b, then the pressure mean removed."""
    from scipy.sparse.linalg import spsolve
    Z = null_basis(N)
    Zs = sp.csr_matrix(Z)
    w = spsolve((L + Zs @ Zs.T).tocsc(), b - Z @ (Z.T @ b))
    return project(w, N)


# ---------------------------------------------------------------------------------- transfers
def prolong_velocity(Nc):
    """RT0 prolongation on the unknowns: the periodic P_u with the wall faces (zero) removed."""
    Nf = 2 * Nc
    P = transfer.prolong_velocity(Nc)
    vf = interior(Nf)[: 2 * Nf * Nf - 2 * Nf]
    vc = interior(Nc)[: 2 * Nc * Nc - 2 * Nc]
    return P[vf][:, vc].tocsr()


def restrict_velocity(Nc):
    return (prolong_velocity(Nc).T / 4.0).tocsr()


def prolong_pressure(Nc):
    """Bilinear from the four nearest coarse centres (9/16, 3/16, 3/16, 1/16), with a neighbour
    outside the domain replaced by the cell itself (reflection across the wall)."""
    Nf = 2 * Nc
    rows, cols, vals = [], [], []
    for jf in range(Nf):
        for i_f in range(Nf):
            I, J = i_f // 2, jf // 2
            si = 1 if i_f % 2 else -1
            sj = 1 if jf % 2 else -1
            I2 = I + si if 0 <= I + si < Nc else I
            J2 = J + sj if 0 <= J + sj < Nc else J
            r = jf * Nf + i_f
            for (ci, cj, w) in ((I, J, 9.0 / 16.0), (I2, J, 3.0 / 16.0), (I, J2, 3.0 / 16.0), (I2, J2, 1.0 / 16.0)):
                rows.append(r)
                cols.append(cj * Nc + ci)
                vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(Nf * Nf, Nc * Nc))


def restrict_pressure(Nc):
    return transfer.restrict_p(Nc)


def prolong(Nc):
    return sp.block_diag([prolong_velocity(Nc), prolong_pressure(Nc)], format="csr")


def restrict(Nc):
    return sp.block_diag([restrict_velocity(Nc), restrict_pressure(Nc)], format="csr")


# ------------------------------------------------------------------------------- smoother, cycle
def vanka_patch_dofs(N):
    """Per cell: the cell's faces that are unknowns and its pressure, as indices into the unknown
    vector, with the weights 1/2 (faces) and 1 (pressure).  Returns a list of (dofs, weights)."""
    n = N * N
    pos = -np.ones(3 * n, dtype=np.int64)
    pos[interior(N)] = np.arange(3 * n - 2 * N)
    out = []
    for j in range(N):
        for i in range(N):
            cand = [cell_index(N, i, j), cell_index(N, i + 1, j), n + cell_index(N, i, j), n + cell_index(N, i, j + 1)]
            d = [int(pos[c]) for c in cand if pos[c] >= 0]
            wts = [0.5] * len(d)
            d.append(int(pos[2 * n + cell_index(N, i, j)]))
            wts.append(1.0)
            out.append((np.array(d), np.array(wts)))
    return out


def vanka_sweep(L, patches, factors, x, b, omega):
    """x <- x + omega sum_c W_c R_c^T L_c^{-1} R_c (b - L x) over the cell patches."""
    r = b - L @ x
    dx = np.zeros_like(x)
    for (d, wts), Lc in zip(patches, factors):
        dx[d] += wts * np.linalg.solve(Lc, r[d])
    return x + omega * dx


class Hierarchy:
    """Levels N_l = n_min 2^l of the cavity; Galerkin coarse IB operator R_u B P_u; per-cell additive
    Vanka (omega = 0.8) or the SC smoother; exact coarsest solve (pseudo-inverse with the pressure
    constant as its kernel); Alg. 1 V-cycle from a zero guess."""

    def __init__(self, N, rho, mu, dt, X, edges, kappa, n_min=8, smoother="vanka", omega=None, nu1=2, nu2=2):
        lmax = int(round(np.log2(N // n_min)))
        if n_min * 2 ** lmax != N:
            raise ValueError("N must be n_min * 2^k")
        self.smoother = smoother
        self.omega = (0.8 if smoother == "vanka" else 1.0) if omega is None else omega
        self.nu1, self.nu2 = nu1, nu2
        Bs = [None] * (lmax + 1)
        Bs[lmax] = ib_operator(N, X, edges, kappa)
        self.P = [None] * (lmax + 1)
        self.R = [None] * (lmax + 1)
        for l in range(lmax, 0, -1):
            Nc = n_min * 2 ** (l - 1)
            self.P[l], self.R[l] = prolong(Nc), restrict(Nc)
            Bs[l - 1] = (restrict_velocity(Nc) @ Bs[l] @ prolong_velocity(Nc)).tocsr()
        self.levels = []
        for l in range(lmax + 1):
            Nl = n_min * 2 ** l
            lev = type("Level", (), {})()
            lev.N = Nl
            lev.A = momentum(Nl, rho, mu, dt)
            lev.G, lev.D = gradient(Nl), divergence(Nl)
            lev.AIB = (lev.A - dt * Bs[l]).tocsr()
            lev.L = sp.bmat([[lev.AIB, lev.G], [-lev.D, None]], format="csr")
            if l > 0 and smoother == "vanka":
                lev.patches = vanka_patch_dofs(Nl)
                Ld = lev.L.tocsr()
                lev.factors = [Ld[d][:, d].toarray() for d, _ in lev.patches]
            elif l > 0:
                lev.dA = lev.AIB.diagonal()
                PA, PM, lev.dM = smoothers.sc_preconditioners(lev.AIB, lev.G, lev.D, lev.dA, "jacobi")
                lev.lamA = smoothers.power_max(lambda z, A=lev.AIB: A @ z, PA, lev.AIB.shape[0], 10)
                Ainv = lambda q, A=lev.AIB, lam=lev.lamA: smoothers.chebyshev(lambda z: A @ z, PA, q, lam, 2)
                lev.lamM = smoothers.power_max(lambda q, lv=lev: lv.D @ Ainv(lv.G @ q), PM, Nl * Nl, 10)
            self.levels.append(lev)
        L0 = self.levels[0].L.toarray()
        Z = null_basis(n_min)
        self.coarse_pinv = np.linalg.inv(L0 + Z @ Z.T) - Z @ Z.T
        self.lmax = lmax

    def smooth(self, l, x, b, sweeps):
        lev = self.levels[l]
        for _ in range(sweeps):
            if self.smoother == "vanka":
                x = vanka_sweep(lev.L, lev.patches, lev.factors, x, b, self.omega)
            else:
                x = smoothers.sc_sweep(lev.L, lev.G, lev.D, lev.AIB, lev.dA, lev.dM, lev.lamA, lev.lamM, x, b,
                                       self.omega, 2)
        return x

    def mg(self, l, w, b):
        if l == 0:
            return self.coarse_pinv @ b
        lev = self.levels[l]
        w = self.smooth(l, w, b, self.nu1)
        rc = self.R[l] @ (b - lev.L @ w)
        w = w + self.P[l] @ self.mg(l - 1, np.zeros_like(rc), rc)
        return self.smooth(l, w, b, self.nu2)

    def vcycle(self, b):
        return self.mg(self.lmax, np.zeros_like(b), b)

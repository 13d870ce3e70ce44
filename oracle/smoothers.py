"""Smoothers on one multigrid level (Sec. 3.3).

Additive Vanka (Alg. 2, restricted additive Schwarz, taken with one-cell subdomains as the
per-cell additive Vanka form): the residual is formed once from the incoming iterate; for every
cell c the 5x5 saddle-point patch operator L_c = R_c L R_c^T on the dofs
(u_{i-1/2,j}, u_{i+1/2,j}, v_{i,j-1/2}, v_{i,j+1/2}, p_{i,j}) is solved against R_c r, and the
corrections are weighted (1/2 on the four faces, each shared by two cells, 1 on the pressure)
and summed.  One sweep is x <- x + omega * sum_c W_c R_c^T L_c^{-1} R_c (b - L x).

Schur-complement smoother (Eqs. fact-Stokes-IB and approx-fact-Stokes-IB):
    y  = At^{-1} r_u,   dp = Mt^{-1}(r_p + D y),   du = y - At^{-1}(G dp),   x <- x + omega (du, dp)
At^{-1}: a fixed number of Chebyshev iterations on A_IB with a point-relaxation preconditioner;
Mt^{-1}: a fixed number of Chebyshev iterations on D At^{-1} G preconditioned by point relaxation
on the sparse approximate Schur complement Mh = D diag(A_IB)^{-1} G.  The paper relaxes with
Gauss-Seidel.  Two relaxations are provided:
- "jacobi": the diagonal inverse (every level is one parallel pass);
- "sgs": one symmetric multicolour Gauss-Seidel sweep from a zero guess.  The dofs are coloured
  red-black by (i + j) mod 2 (u and v faces alike, and the cells of Mh), which separates every pair
  of unknowns coupled by the five-point stencils.  A colour pass updates its colour as
  z_c <- z_c + (r - Op z)_c / diag_c with Op z taken from the iterate at the start of the pass; the
  sweep runs the colours forward then backward (0, 1, 1, 0), so the preconditioner is symmetric.
  For Mh, and for A_IB rows without IB couplings, this is exactly Gauss-Seidel in red-black order;
  the IB couplings [S K J] also link faces of one colour, and those enter from the start of the
  pass.

Restricted additive Schwarz over boxes (Alg. 2 with b x b subdomains and overlap o, the paper's
Vanka-type smoother): every box solves its local saddle-point problem (all faces of its extended
cells and their pressures) on the current residual; each dof takes the correction of the box that
owns it (no weights: the owned sets partition the dofs).

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
import scipy.sparse as sp

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


def ras_boxes(N, b, o):
    """Dof lists of the box subdomains of the restricted additive Schwarz smoother (Sec. 3.3, RAS).

    The cells are tiled by b x b core boxes, box (I, J) covering cells I b .. I b + b - 1 by
    J b .. J b + b - 1; its subdomain extends the core by o cells on each side (periodic), e = b + 2o
    cells wide.  The subdomain's dofs are every face of its e x e cells and their pressures:
        u(i, j), i = I b - o .. I b + b + o (e + 1 columns), j over the e rows,
        v(i, j), i over the e columns, j = J b - o .. J b + b + o (e + 1 rows),
        p(i, j) over the e x e cells,
    in that order, row-major within each.  A dof is owned by the box whose core holds it: u(i, j) and
    v(i, j) belong to cell (i, j) (its left and bottom faces), p(i, j) to the cell; every dof has one
    owner.  Returns [(dofs, owned_mask)] over the boxes, row-major in (J, I)."""
    if N % b or b + 2 * o + 1 > N:
        raise ValueError("b must divide N and the subdomain must not wrap onto itself")
    n, e = N * N, b + 2 * o
    out = []
    for J in range(N // b):
        for I in range(N // b):
            i0, j0 = I * b - o, J * b - o
            core_i = lambda ii: I * b <= ii < I * b + b
            core_j = lambda jj: J * b <= jj < J * b + b
            dofs, own = [], []
            for jj in range(j0, j0 + e):
                for ii in range(i0, i0 + e + 1):
                    dofs.append(cell_index(N, ii, jj))
                    own.append(core_i(ii) and core_j(jj))
            for jj in range(j0, j0 + e + 1):
                for ii in range(i0, i0 + e):
                    dofs.append(n + cell_index(N, ii, jj))
                    own.append(core_i(ii) and core_j(jj))
            for jj in range(j0, j0 + e):
                for ii in range(i0, i0 + e):
                    dofs.append(2 * n + cell_index(N, ii, jj))
                    own.append(core_i(ii) and core_j(jj))
            out.append((np.array(dofs), np.array(own)))
    return out


def ras_factors(L, boxes):
    """LU factors of every subdomain operator L_k = R_k L R_k^T (dense)."""
    import scipy.linalg as sla
    Ld = L.tocsr()
    return [sla.lu_factor(Ld[d][:, d].toarray()) for d, _ in boxes]


def ras_wraps(N, b, o):
    """True where a b x b box with overlap o has no subdomain on an N x N level: b does not divide N, or
    the e + 1 = b + 2o + 1 face columns of a subdomain would wrap onto themselves."""
    return N % b != 0 or b + 2 * o + 1 > N


def exact_level_sweep(L, pinv, x, b, omega):
    """The RAS sweep's reading on a level too small for its boxes (`ras_wraps`): the box, clipped to the
    periodic level, is the whole level, so its local solve is the exact level solve; the level operator
    is singular (its kernel: the constant pressure, and the constant velocities when rho = 0), and the
    solve is the gauge-fixed pseudo-inverse, as for the coarsest level:
        x <- x + omega L^+ (b - L x)."""
    return x + omega * (pinv @ (b - L @ x))


def ras_sweep(L, boxes, factors, x, b, omega):
    """x <- x + omega sum_k Rt_k^T L_k^{-1} R_k (b - L x): every subdomain solves its local problem on
    the residual, and each dof takes the correction of the box that owns it."""
    import scipy.linalg as sla
    r = b - L @ x
    dx = np.zeros_like(x)
    for (d, own), f in zip(boxes, factors):
        delta = sla.lu_solve(f, r[d])
        dx[d[own]] = delta[own]
    return x + omega * dx


def hash_vector(n):
    """Deterministic start vector: Knuth's multiplicative hash of (k+1), mapped to [-1/2, 1/2)."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    return ((k * np.uint64(2654435761)) % np.uint64(2 ** 32)).astype(np.float64) / 2.0 ** 32 - 0.5


def _as_prec(prec):
    """A preconditioner given as a vector is the diagonal scaling by it; a callable is applied."""
    if callable(prec):
        return prec
    return lambda r: prec * r


def power_max(apply_op, prec, n, iters):
    """Estimate of the largest eigenvalue of P Op (P = diag(prec), or the callable prec):
    ||w|| after `iters` normalised steps."""
    P = _as_prec(prec)
    v = hash_vector(n)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = P(apply_op(v))
        lam = np.linalg.norm(w)
        v = w / lam
    return lam


def chebyshev(apply_op, prec, b, lam_max, iters, lo=0.1, hi=1.1):
    """`iters` Chebyshev iterations for Op x = b from x_0 = 0 with preconditioner P (diag(prec), or
    the callable prec)."""
    P = _as_prec(prec)
    lmin, lmax = lo * lam_max, hi * lam_max
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = b.copy()
    d = P(r) / theta
    x = np.zeros_like(b)
    for k in range(iters):
        x = x + d
        if k == iters - 1:
            break
        r = r - apply_op(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * P(r)
        rho = rho_new
    return x


def rb_colours(N, fields):
    """Red-black colour (i + j) mod 2 of every dof of `fields` stacked N x N fields, row-major [j][i]."""
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return np.tile(((i + j) % 2).ravel(), fields)


def sgs_multicolour(Op, diag, colours, r):
    """One symmetric multicolour Gauss-Seidel sweep for Op z = r from z = 0: colour passes 0, 1, 1, 0,
    each z_c <- z_c + (r - Op z)_c / diag_c with Op z from the start of the pass."""
    z = np.zeros_like(r)
    for c in (0, 1, 1, 0):
        sel = colours == c
        res = r - Op @ z
        z[sel] = z[sel] + res[sel] / diag[sel]
    return z


def sc_preconditioners(AIB, G, D, dA, relax):
    """(P_A, P_M): the point relaxations of A_IB and of Mh = D diag(A_IB)^{-1} G used inside the
    Chebyshev iterations; diag(Mh) is returned as the third value."""
    Mh = (D @ sp.diags(1.0 / dA) @ G).tocsr()
    dM = Mh.diagonal()
    if relax == "jacobi":
        return 1.0 / dA, 1.0 / dM, dM
    if relax != "sgs":
        raise ValueError("relax must be 'jacobi' or 'sgs'")
    N = int(round(np.sqrt(G.shape[1])))
    cu, cp = rb_colours(N, 2), rb_colours(N, 1)
    return (lambda q: sgs_multicolour(AIB, dA, cu, q)), (lambda q: sgs_multicolour(Mh, dM, cp, q)), dM


def sc_apply(r, nu, Ainv, Minv, G, D):
    """Approximate block-factorised inverse applied to r = (r_u, r_p)."""
    y = Ainv(r[:nu])
    dp = Minv(r[nu:] + D @ y)
    du = y - Ainv(G @ dp)
    return np.concatenate([du, dp])


def sc_sweep(L, G, D, AIB, dA, dM, lamA, lamM, x, b, omega, cheb_iters, lo=0.1, hi=1.1, relax="jacobi"):
    nu = G.shape[0]
    PA, PM, _ = sc_preconditioners(AIB, G, D, dA, relax)

    def Ainv(q):
        return chebyshev(lambda z: AIB @ z, PA, q, lamA, cheb_iters, lo, hi)

    def Mop(q):
        return D @ Ainv(G @ q)

    def Minv(q):
        return chebyshev(Mop, PM, q, lamM, cheb_iters, lo, hi)

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

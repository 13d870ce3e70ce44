"""Lagrangian-Eulerian coupling and the spring operator (Sec. 2.2, Appendix "Lagrangian discretization"
and "Lagrangian-Eulerian interaction").

Interpolation (Appendix, discrete velocity interpolation): with face positions x_f,
    U_l = sum_f u_f delta_h(x_f - X_l) h^2 = sum_f u_f phi((x_f - X_l)/h) phi((y_f - Y_l)/h),
so J[l, f] = phi(.) phi(.) and U = J u, one matrix per velocity component.
Spreading (Appendix, discrete force spreading): the spring force F_l is a force (not a force
density), so the spread force density is f_f = sum_l F_l delta_h(x_f - X_l), i.e. S = J^T / h^2.
With the h^2-weighted grid inner product this is the discrete adjointness S = J^* of the paper.
Springs (Eq. F-lin-functional and its finite-difference form): zero-rest-length links give
F_a = sum_{e=(a,b)} kappa_e (X_b - X_a), componentwise; K = -sum_e kappa_e (e_a - e_b)(e_a - e_b)^T.
For fiber links this is the paper's alpha * D_s1 D_s1 X with kappa_e = alpha / Delta s_1.

Pinned by: brute-force dense J (minimum-image distances) equals the local 4x4 construction;
<S F, u>_h = <F, J u>; partition of unity of every row of J; K (translation) = 0, K symmetric
negative semidefinite, brute force on a three-marker ring.
"""
import numpy as np
import scipy.sparse as sp

from .peskin import phi

# offsets of face positions in units of h: x-faces at (i, j+1/2), y-faces at (i+1/2, j)
FACE_OFFSET = {0: (0.0, 0.5), 1: (0.5, 0.0)}


def interp_matrix(N, X, comp):
    """J for velocity component comp (0: u on x-faces, 1: v on y-faces), sparse (M x N^2)."""
    h = 1.0 / N
    M = X.shape[0]
    if M == 0:
        return sp.csr_matrix((0, N * N))
    ox, oy = FACE_OFFSET[comp]
    sx = X[:, 0] / h - ox
    sy = X[:, 1] / h - oy
    i0 = np.floor(sx).astype(np.int64) - 1
    j0 = np.floor(sy).astype(np.int64) - 1
    rows, cols, vals = [], [], []
    for a in range(4):
        wx = phi((i0 + a) - sx)
        for b in range(4):
            wy = phi((j0 + b) - sy)
            rows.append(np.arange(M))
            cols.append(np.mod(j0 + b, N) * N + np.mod(i0 + a, N))
            vals.append(wx * wy)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(M, N * N))


def interp_matrix_bruteforce(N, X, comp):
    """Dense J from minimum-image distances to every face (tiny grids only)."""
    h = 1.0 / N
    ox, oy = FACE_OFFSET[comp]
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    xf = ((i + ox) * h).ravel()
    yf = ((j + oy) * h).ravel()
    J = np.zeros((X.shape[0], N * N))
    for l in range(X.shape[0]):
        dx = xf - X[l, 0]
        dy = yf - X[l, 1]
        dx -= np.round(dx)
        dy -= np.round(dy)
        J[l] = phi(dx / h) * phi(dy / h)
    return J


def spread_matrix(N, X, comp):
    """S = J^T / h^2 for one component (N^2 x M)."""
    h = 1.0 / N
    return (interp_matrix(N, X, comp).T / (h * h)).tocsr()


def stiffness(M, edges, kappa):
    """K = -sum_e kappa_e (e_a - e_b)(e_a - e_b)^T  (M x M), applied to each component."""
    if edges.shape[0] == 0:
        return sp.csr_matrix((M, M))
    a = edges[:, 0].astype(np.int64)
    b = edges[:, 1].astype(np.int64)
    k = np.asarray(kappa, dtype=np.float64)
    rows = np.concatenate([a, b, a, b])
    cols = np.concatenate([a, b, b, a])
    vals = np.concatenate([-k, -k, k, k])
    return sp.csr_matrix((vals, (rows, cols)), shape=(M, M))


def spring_force(X, edges, kappa):
    """F = K X, by looping over the springs (reference form of Eq. F-lin-functional)."""
    F = np.zeros_like(X)
    for (a, b), k in zip(edges, kappa):
        F[a] += k * (X[b] - X[a])
        F[b] += k * (X[a] - X[b])
    return F


def ib_operator(N, X, edges, kappa):
    """S K J on the velocity faces (2 N^2 x 2 N^2, block-diagonal per component)."""
    K = stiffness(X.shape[0], edges, kappa)
    blocks = []
    for c in (0, 1):
        J = interp_matrix(N, X, c)
        S = spread_matrix(N, X, c)
        blocks.append((S @ K @ J).tocsr())
    return sp.block_diag(blocks, format="csr")


def spread_force(N, X, F):
    """f = S F on both components, F (M x 2) -> (2 N^2,)."""
    return np.concatenate([spread_matrix(N, X, c) @ F[:, c] for c in (0, 1)])


def interp_velocity(N, X, w):
    """U = J u for w = [u | v | ...] -> (M x 2)."""
    n = N * N
    return np.stack([interp_matrix(N, X, 0) @ w[:n], interp_matrix(N, X, 1) @ w[n:2 * n]], axis=1)

"""Periodic staggered (MAC) grid operators as scipy.sparse matrices (Appendix, "Eulerian discretization").

Unknowns on an N x N periodic grid, h = 1/N, every block row-major [j][i]:
  u[j][i] on the x-face (i-1/2, j) of cell (i, j)  -> index j*N + i of the u block
  v[j][i] on the y-face (i, j-1/2) of cell (i, j)  -> index j*N + i of the v block
  p[j][i] at the centre of cell (i, j)
Standard second-order differences:
  (Lap q)_{i,j} = (q_{i+1,j} + q_{i-1,j} + q_{i,j+1} + q_{i,j-1} - 4 q_{i,j}) / h^2
  (G p)^x_{i-1/2,j} = (p_{i,j} - p_{i-1,j}) / h,   (G p)^y_{i,j-1/2} = (p_{i,j} - p_{i,j-1}) / h
  (D u)_{i,j} = (u_{i+1/2,j} - u_{i-1/2,j} + v_{i,j+1/2} - v_{i,j-1/2}) / h
  A = (rho/dt) I - mu Lap   on each velocity component (Eq. system-impib)

Pinned by: D = -G^T; the Fourier symbols of Lap, G, D on periodic modes (tests/test_oracle_pins.py).
"""
import numpy as np
import scipy.sparse as sp


def cell_index(N, i, j):
    return (np.mod(j, N) * N + np.mod(i, N)).astype(np.int64)


def _grid(N):
    j, i = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    return i.ravel(), j.ravel()


def laplacian(N):
    h = 1.0 / N
    i, j = _grid(N)
    row = cell_index(N, i, j)
    rows, cols, vals = [], [], []
    for di, dj, w in ((0, 0, -4.0), (1, 0, 1.0), (-1, 0, 1.0), (0, 1, 1.0), (0, -1, 1.0)):
        rows.append(row)
        cols.append(cell_index(N, i + di, j + dj))
        vals.append(np.full(row.size, w / (h * h)))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N * N, N * N))


def gradient(N):
    """G: pressure (N^2) -> velocity faces (2 N^2)."""
    h = 1.0 / N
    n = N * N
    i, j = _grid(N)
    f = cell_index(N, i, j)
    rows = np.concatenate([f, f, n + f, n + f])
    cols = np.concatenate([cell_index(N, i, j), cell_index(N, i - 1, j),
                           cell_index(N, i, j), cell_index(N, i, j - 1)])
    vals = np.concatenate([np.full(n, 1.0 / h), np.full(n, -1.0 / h),
                           np.full(n, 1.0 / h), np.full(n, -1.0 / h)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * n, n))


def divergence(N):
    """D: velocity faces (2 N^2) -> cells (N^2)."""
    h = 1.0 / N
    n = N * N
    i, j = _grid(N)
    c = cell_index(N, i, j)
    rows = np.concatenate([c, c, c, c])
    cols = np.concatenate([cell_index(N, i + 1, j), cell_index(N, i, j),
                           n + cell_index(N, i, j + 1), n + cell_index(N, i, j)])
    vals = np.concatenate([np.full(n, 1.0 / h), np.full(n, -1.0 / h),
                           np.full(n, 1.0 / h), np.full(n, -1.0 / h)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, 2 * n))


def momentum(N, rho, mu, dt):
    """A = (rho/dt) I - mu Lap on both velocity components (2 N^2 x 2 N^2)."""
    n = N * N
    Ac = (rho / dt) * sp.identity(n, format="csr") - mu * laplacian(N)
    return sp.block_diag([Ac, Ac], format="csr")

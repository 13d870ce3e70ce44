"""Inter-level transfer operators (Sec. 3.2, "Prolongation and restriction"), refinement ratio 2.

Velocity prolongation P_u is lowest-order Raviart-Thomas interpolation: linear in the direction
normal to a face, constant in the tangential direction.  For x-faces, fine face (i, j) of the
fine grid (N_f = 2 N_c) takes
    i even:  u_c(i/2, floor(j/2))
    i odd :  (u_c((i-1)/2, floor(j/2)) + u_c((i+1)/2, floor(j/2))) / 2
and symmetrically for y-faces.  Velocity restriction is the adjoint of P_u in the h^2-weighted
grid inner product, R_u = (h_f^2 / h_c^2) P_u^T = P_u^T / 4 (it keeps constants).
Pressure prolongation is linear (bilinear from the four nearest coarse centres, weights
9/16, 3/16, 3/16, 1/16); pressure restriction is the average of the four fine cells.

Pinned by: R_u 1 = 1; D_f P_u = (piecewise-constant injection) D_c; R_u G_f = G_c R_p;
P_p reproduces coarse fields that are linear in x and y away from the periodic seam.
"""
import numpy as np
import scipy.sparse as sp

from .mac import cell_index


def _fine_grid(Nc):
    Nf = 2 * Nc
    j, i = np.meshgrid(np.arange(Nf), np.arange(Nf), indexing="ij")
    return Nf, i.ravel(), j.ravel()


def prolong_u(Nc):
    """P for x-face velocity (Nf^2 x Nc^2)."""
    Nf, i, j = _fine_grid(Nc)
    row = cell_index(Nf, i, j)
    J = j // 2
    even = (i % 2) == 0
    rows = [row[even]]
    cols = [cell_index(Nc, i[even] // 2, J[even])]
    vals = [np.ones(even.sum())]
    odd = ~even
    for off in (0, 1):
        rows.append(row[odd])
        cols.append(cell_index(Nc, (i[odd] - 1) // 2 + off, J[odd]))
        vals.append(np.full(odd.sum(), 0.5))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(Nf * Nf, Nc * Nc))


def prolong_v(Nc):
    """P for y-face velocity (Nf^2 x Nc^2)."""
    Nf, i, j = _fine_grid(Nc)
    row = cell_index(Nf, i, j)
    I = i // 2
    even = (j % 2) == 0
    rows = [row[even]]
    cols = [cell_index(Nc, I[even], j[even] // 2)]
    vals = [np.ones(even.sum())]
    odd = ~even
    for off in (0, 1):
        rows.append(row[odd])
        cols.append(cell_index(Nc, I[odd], (j[odd] - 1) // 2 + off))
        vals.append(np.full(odd.sum(), 0.5))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(Nf * Nf, Nc * Nc))


def prolong_p(Nc):
    """Bilinear cell-centred prolongation (Nf^2 x Nc^2)."""
    Nf, i, j = _fine_grid(Nc)
    row = cell_index(Nf, i, j)
    I, J = i // 2, j // 2
    si = np.where(i % 2 == 0, -1, 1)   # neighbour side in x
    sj = np.where(j % 2 == 0, -1, 1)
    rows, cols, vals = [], [], []
    for di, dj, w in ((0, 0, 9 / 16), (1, 0, 3 / 16), (0, 1, 3 / 16), (1, 1, 1 / 16)):
        rows.append(row)
        cols.append(cell_index(Nc, I + di * si, J + dj * sj))
        vals.append(np.full(row.size, w))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(Nf * Nf, Nc * Nc))


def restrict_p(Nc):
    """Average of the four fine cells (Nc^2 x Nf^2)."""
    Nf = 2 * Nc
    J, I = np.meshgrid(np.arange(Nc), np.arange(Nc), indexing="ij")
    I, J = I.ravel(), J.ravel()
    row = cell_index(Nc, I, J)
    rows, cols, vals = [], [], []
    for di in (0, 1):
        for dj in (0, 1):
            rows.append(row)
            cols.append(cell_index(Nf, 2 * I + di, 2 * J + dj))
            vals.append(np.full(row.size, 0.25))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(Nc * Nc, Nf * Nf))


def prolong_velocity(Nc):
    return sp.block_diag([prolong_u(Nc), prolong_v(Nc)], format="csr")


def restrict_velocity(Nc):
    return (0.25 * prolong_velocity(Nc).T).tocsr()


def prolong(Nc):
    """Block prolongation on [u | v | p]."""
    return sp.block_diag([prolong_u(Nc), prolong_v(Nc), prolong_p(Nc)], format="csr")


def restrict(Nc):
    """Block restriction on [u | v | p]."""
    return sp.block_diag([0.25 * prolong_u(Nc).T, 0.25 * prolong_v(Nc).T, restrict_p(Nc)], format="csr")

"""Adjoint of the Stokes-IB solve and gradients with respect to spring stiffness and marker positions.

The paper has no differentiation; this restates the discrete adjoint of its Eq. matrix-impib.
For a loss l(w) of the gauge-fixed solution w = (u, p) of L(X, kappa) w = b(X, kappa):
  * adjoint: L^T lambda = dl/dw; L is symmetric, so lambda solves the same system (gauge-fixed,
    adjoint right-hand side projected like any right-hand side);
  * dl = lambda_u^T [ d(S K X^n) + dt d(S K J) u ] with u held fixed.  With S = J^T/h^2 this is
    d[ Lam^T K Y ] where Lam = J lambda_u / h^2 and Y = a X^n + dt U, U = J u
    (a = 1 when the right-hand side carries S K X^n, else 0):
      dl/dkappa_e = -(Lam_a - Lam_b) . (Y_a - Y_b)
      dl/dX_l^d  = sum_c (d_d Lam_l^c) (K Y)_l^c + a (K Lam)_l^d + dt sum_c (K Lam)_l^c d_d U_l^c
    with d_d J^c_{l,f} = -(1/h) phi'(r_x) phi(r_y) (d = x) or -(1/h) phi(r_x) phi'(r_y) (d = y);
  * dl/dg = lambda_u.

Pinned by: central finite differences of the loss of direct solves (tests/test_oracle_adjoint.py).
"""
import numpy as np
import scipy.sparse as sp

from . import ib, system
from .peskin import dphi, phi


def grad_interp_matrix(N, X, comp, d):
    """d J^c / d X^d as a sparse (M x N^2) matrix (row l holds the derivative w.r.t. X_l)."""
    h = 1.0 / N
    M = X.shape[0]
    ox, oy = ib.FACE_OFFSET[comp]
    sx = X[:, 0] / h - ox
    sy = X[:, 1] / h - oy
    i0 = np.floor(sx).astype(np.int64) - 1
    j0 = np.floor(sy).astype(np.int64) - 1
    rows, cols, vals = [], [], []
    for a in range(4):
        rx = (i0 + a) - sx
        for b in range(4):
            ry = (j0 + b) - sy
            if d == 0:
                v = -dphi(rx) * phi(ry) / h
            else:
                v = -phi(rx) * dphi(ry) / h
            rows.append(np.arange(M))
            cols.append(np.mod(j0 + b, N) * N + np.mod(i0 + a, N))
            vals.append(v)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(M, N * N))


def gradients(prob, w, lam, add_SKXn=True):
    """(dl/dkappa (E,), dl/dX (M,2), dl/dg (2N^2,)) from the forward solution w and adjoint lam."""
    N, n = prob.N, prob.N * prob.N
    h = 1.0 / N
    s = prob.structure
    M = s.M
    K = ib.stiffness(M, s.edges, s.kappa)
    a = 1.0 if add_SKXn else 0.0
    Lam = np.zeros((M, 2))
    U = np.zeros((M, 2))
    for c in (0, 1):
        J = ib.interp_matrix(N, s.X, c)
        Lam[:, c] = J @ lam[c * n:(c + 1) * n] / (h * h)
        U[:, c] = J @ w[c * n:(c + 1) * n]
    Y = a * s.X + prob.dt * U
    ea, eb = s.edges[:, 0], s.edges[:, 1]
    dkappa = -np.sum((Lam[ea] - Lam[eb]) * (Y[ea] - Y[eb]), axis=1)
    KY = K @ Y
    KLam = K @ Lam
    dX = a * KLam.copy()
    for d in (0, 1):
        for c in (0, 1):
            dJ = grad_interp_matrix(N, s.X, c, d)
            dLam = dJ @ lam[c * n:(c + 1) * n] / (h * h)
            dU = dJ @ w[c * n:(c + 1) * n]
            dX[:, d] += dLam * KY[:, c] + prob.dt * KLam[:, c] * dU
    dg = lam[:2 * n].copy()
    return dkappa, dX, dg


def velocity_loss(w, target, n):
    diff = w[:2 * n] - target[:2 * n]
    return float(diff @ diff)


def solve(prob, add_SKXn=True):
    """Gauge-fixed direct solution w of the problem."""
    L = system.operator_of(prob)
    b = system.rhs(prob, add_SKXn)
    w, _ = system.solve_direct(L, b, prob.N, prob.rho)
    return system.project(w, prob.N, prob.rho)


def loss_and_gradients(prob, target, add_SKXn=True):
    """Loss ||u - u_target||^2 over the velocity faces and its gradients, all by direct solves."""
    N, n = prob.N, prob.N * prob.N
    L = system.operator_of(prob)
    b = system.rhs(prob, add_SKXn)
    w, _ = system.solve_direct(L, b, N, prob.rho)
    w = system.project(w, N, prob.rho)
    rhs_adj = np.zeros(3 * n)
    rhs_adj[:2 * n] = 2.0 * (w[:2 * n] - target[:2 * n])
    rhs_adj = system.project(rhs_adj, N, prob.rho)
    lam, _ = system.solve_direct(L, rhs_adj, N, prob.rho)
    lam = system.project(lam, N, prob.rho)
    return velocity_loss(w, target, n), w, lam, gradients(prob, w, lam, add_SKXn)

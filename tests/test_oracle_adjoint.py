"""Pins of the oracle's adjoint gradients against central finite differences of direct solves."""
import numpy as np
import pytest

from oracle import adjoint, system
from paper_1612_02208_gb300 import inputs as I


def _problem(N, rho=0.0):
    prob = I.thin_ellipse_loguniform(N)
    if rho:
        prob.rho, prob.mu, prob.dt = rho, 1e-2, 1e-3
    return prob


def _target(prob):
    other = I.thin_ellipse_loguniform(prob.N, seed_kappa=30)
    other.rho, other.mu, other.dt = prob.rho, prob.mu, prob.dt
    return adjoint.solve(other)


def _loss(prob, target, add):
    w = adjoint.solve(prob, add)
    return adjoint.velocity_loss(w, target, prob.N * prob.N)


@pytest.mark.parametrize("add,rho", [(True, 0.0), (False, 0.0), (True, 1.0)])
def test_gradients_match_central_differences(add, rho):
    prob = _problem(16, rho)
    target = _target(prob)
    loss, w, lam, (dk, dX, dg) = adjoint.loss_and_gradients(prob, target, add)
    rng = np.random.default_rng(300)
    s = prob.structure
    for _ in range(4):
        # kappa direction (relative)
        dir_k = rng.standard_normal(s.E) * s.kappa
        eps = 1e-6
        p1 = _problem(16, rho); p1.structure.kappa = s.kappa + eps * dir_k
        p2 = _problem(16, rho); p2.structure.kappa = s.kappa - eps * dir_k
        fd = (_loss(p1, target, add) - _loss(p2, target, add)) / (2 * eps)
        assert abs(fd - dk @ dir_k) < 1e-6 * (abs(fd) + 1e-3 * loss), (fd, dk @ dir_k)
        # marker direction
        dir_x = rng.standard_normal(s.X.shape) * 1e-2
        eps = 1e-5
        p1 = _problem(16, rho); p1.structure.X = s.X + eps * dir_x
        p2 = _problem(16, rho); p2.structure.X = s.X - eps * dir_x
        fd = (_loss(p1, target, add) - _loss(p2, target, add)) / (2 * eps)
        assert abs(fd - np.sum(dX * dir_x)) < 1e-5 * (abs(fd) + 1e-3 * loss), (fd, np.sum(dX * dir_x))
        # forcing direction
        dir_g = np.zeros(3 * 256)
        dir_g[:512] = rng.standard_normal(512)
        eps = 1e-4
        p1 = _problem(16, rho); p1.g = prob.g + eps * dir_g
        p2 = _problem(16, rho); p2.g = prob.g - eps * dir_g
        fd = (_loss(p1, target, add) - _loss(p2, target, add)) / (2 * eps)
        assert abs(fd - dg @ dir_g[:512]) < 1e-7 * (abs(fd) + loss), (fd, dg @ dir_g[:512])

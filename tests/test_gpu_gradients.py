"""Gradients of the differentiable solve (adjoint through the same V-cycle) against central finite
differences of the forward solve, on 16 seeded random directions, at the 256 x 256 size of the
log-uniform-stiffness workload, for the FP64 and the FP32-preconditioned solver."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402
from paper_1612_02208_gb300.autograd import stokes_ib_solve  # noqa: E402


def _setup(N, fp32):
    prob = I.thin_ellipse_loguniform(N)
    target_prob = I.thin_ellipse_loguniform(N, seed_kappa=30)
    S = sib.solver_for(target_prob, rtol=1e-13, vcycle_fp32=fp32)
    ut = S.solve(torch.as_tensor(target_prob.g, device="cuda")).detach()
    S.set_options(rtol=1e-13, vcycle_fp32=fp32)
    st = prob.structure
    g = torch.as_tensor(prob.g, device="cuda")
    kap = torch.as_tensor(st.kappa, device="cuda")
    X = torch.as_tensor(st.X, device="cuda")
    E = torch.as_tensor(st.edges, device="cuda")
    return prob, S, g, kap, X, E, ut


def _loss(S, g, kap, X, E, ut, n):
    w = stokes_ib_solve(S, g, kap, X, E)
    return ((w[:2 * n] - ut[:2 * n]) ** 2).sum()


@pytest.mark.parametrize("fp32", [0, 1])
def test_autograd_matches_central_differences(fp32):
    N = 256
    n = N * N
    prob, S, g, kap, X, E, ut = _setup(N, fp32)
    kap_p = kap.clone().requires_grad_(True)
    X_p = X.clone().requires_grad_(True)
    g_p = g.clone().requires_grad_(True)
    loss = _loss(S, g_p, kap_p, X_p, E, ut, n)
    loss.backward()
    dk, dX, dg = kap_p.grad, X_p.grad, g_p.grad
    rng = np.random.default_rng(300)
    worst = 0.0
    for _ in range(16):
        vk = torch.as_tensor(rng.standard_normal(kap.shape[0]), device="cuda") * kap
        vX = torch.as_tensor(rng.standard_normal(X.shape) * 1e-2, device="cuda")
        vg = torch.zeros_like(g)
        vg[:2 * n] = torch.as_tensor(rng.standard_normal(2 * n), device="cuda")
        eps = 1e-6
        with torch.no_grad():
            lp = _loss(S, g + eps * vg, kap + eps * vk, X + eps * vX, E, ut, n)
            lm = _loss(S, g - eps * vg, kap - eps * vk, X - eps * vX, E, ut, n)
        fd = float((lp - lm) / (2 * eps))
        ad = float((dk * vk).sum() + (dX * vX).sum() + (dg * vg).sum())
        err = abs(fd - ad) / (abs(fd) + 1e-12 * float(loss.detach()))
        worst = max(worst, err)
    assert worst < 1e-4, worst


def test_autograd_matches_oracle_dense_solve_gradient():
    N = 32
    prob = I.thin_ellipse_loguniform(N)
    target = adjoint.solve(I.thin_ellipse_loguniform(N, seed_kappa=30))
    loss_ref, _, _, (dk_ref, dX_ref, dg_ref) = adjoint.loss_and_gradients(prob, target)
    S = sib.Solver(N)
    S.set_fluid(prob.rho, prob.mu, prob.dt)
    S.set_options(rtol=1e-13)
    st = prob.structure
    g = torch.as_tensor(prob.g, device="cuda").requires_grad_(True)
    kap = torch.as_tensor(st.kappa, device="cuda").requires_grad_(True)
    X = torch.as_tensor(st.X, device="cuda").requires_grad_(True)
    E = torch.as_tensor(st.edges, device="cuda")
    w = stokes_ib_solve(S, g, kap, X, E)
    ut = torch.as_tensor(target, device="cuda")
    loss = ((w[:2 * N * N] - ut[:2 * N * N]) ** 2).sum()
    loss.backward()
    assert abs(float(loss) - loss_ref) < 1e-10 * loss_ref
    for got, ref in ((kap.grad, dk_ref), (X.grad, dX_ref), (g.grad[:2 * N * N], dg_ref)):
        got = got.detach().cpu().numpy()
        assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()

"""Gradients of the differentiable solve (adjoint through the same V-cycle) against central finite
differences of the forward solve, on 16 seeded random directions, at the 256 x 256 size of the
log-uniform-stiffness workload, for the FP64 and the FP32-preconditioned solver; against the oracle's
dense-solve gradient at 32 x 32; and the 1024 x 1024 disk-and-ellipse differentiated solve against the
oracle's residuals and adjoint formula and against central differences."""
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


def test_headline_differentiated_solve_at_full_size():
    """The 1024^2 disk and ellipse (rho = 1, mu = 1e-2, dt = 1e-3, kappa = 1e4, about 3e5 markers), SC in
    its FGMRES-wrapped form, FP32 V-cycle inside FP64 FGMRES, loss ||u - u*||^2 with u* from a solve with
    another seeded forcing:
      * the forward and adjoint solves' reported residuals equal the oracle's matrix-free residuals
        of the returned w and lam, and meet the 1e-8 target;
      * dkappa and dX from sib_grad equal the oracle's adjoint formula evaluated on the GPU's w and lam;
      * central differences of the loss (solves to 1e-11) along four seeded directions in (kappa, X, g)
        match the adjoint gradient."""
    from tests.test_gpu_parity import _oracle_apply
    from oracle import system
    prob = I.disk_and_ellipse_re(1024)
    N, n = prob.N, prob.N * prob.N
    st = prob.structure
    S = sib.solver_for(prob, smoother=sib.SMOOTHER_SC, smooth_krylov=1, vcycle_fp32=1)
    ustar = S.solve(torch.as_tensor(I.forcing(N, 40), device="cuda"))[:2 * n].clone()
    g = torch.as_tensor(prob.g, device="cuda")
    kap = torch.as_tensor(st.kappa, device="cuda")
    X = torch.as_tensor(st.X, device="cuda")
    E = torch.as_tensor(st.edges, device="cuda")
    # forward, adjoint and gradients through the C calls; residuals and gradients against the oracle
    S.set_structure(X, E, kap)
    S.setup()
    w = S.solve(g)
    fwd = S.stats.as_dict()
    adj = torch.zeros_like(w)
    adj[:2 * n] = 2.0 * (w[:2 * n] - ustar)
    lam = S.solve_transpose(adj)
    bwd = S.stats.as_dict()
    dk, dX = S.grad(w, lam)
    wh, lh, ah = w.cpu().numpy(), lam.cpu().numpy(), adj.cpu().numpy()
    b = system.rhs(prob)
    r_fwd = np.linalg.norm(b - _oracle_apply(prob, wh)) / np.linalg.norm(b)
    r_adj = np.linalg.norm(ah - _oracle_apply(prob, lh)) / np.linalg.norm(ah)
    assert fwd["converged"] and bwd["converged"]
    assert abs(r_fwd - fwd["rel_residual"]) <= 1e-6 * r_fwd and r_fwd <= 1.05e-8, (r_fwd, fwd["rel_residual"])
    assert abs(r_adj - bwd["rel_residual"]) <= 1e-6 * r_adj and r_adj <= 1.05e-8, (r_adj, bwd["rel_residual"])
    rk, rX, _ = adjoint.gradients(prob, wh, lh)
    for got, ref in ((dk, rk), (dX, rX)):
        got = got.cpu().numpy()
        assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()
    # central differences through the autograd binding, solves to 1e-11
    S.set_options(rtol=1e-11, max_it=300)
    ut = torch.cat([ustar, torch.zeros(n, dtype=ustar.dtype, device="cuda")])
    kap_p = kap.clone().requires_grad_(True)
    X_p = X.clone().requires_grad_(True)
    g_p = g.clone().requires_grad_(True)
    loss = _loss(S, g_p, kap_p, X_p, E, ut, n)
    loss.backward()
    rng = np.random.default_rng(301)
    for _ in range(4):
        vk = torch.as_tensor(rng.standard_normal(kap.shape[0]), device="cuda") * kap
        vX = torch.as_tensor(rng.standard_normal(X.shape) * 1e-3, device="cuda")
        vg = torch.zeros_like(g)
        vg[:2 * n] = torch.as_tensor(rng.standard_normal(2 * n), device="cuda")
        eps = 1e-6
        with torch.no_grad():
            lp = _loss(S, g + eps * vg, kap + eps * vk, X + eps * vX, E, ut, n)
            lm = _loss(S, g - eps * vg, kap - eps * vk, X - eps * vX, E, ut, n)
        fd = float((lp - lm) / (2 * eps))
        ad = float((kap_p.grad * vk).sum() + (X_p.grad * vX).sum() + (g_p.grad * vg).sum())
        assert abs(fd - ad) <= 1e-4 * abs(fd), (fd, ad)

"""GPU parity of the lid-driven cavity operator (Sec. 5: no-slip walls) against the cavity oracle,
level by level, with the paper's annulus immersed (Galerkin coarse IB operators)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cavity  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402

from tests.test_gpu_parity import TOL32, TOL64, cu, host, rel  # noqa: E402


@pytest.mark.parametrize("rho,mu", [(0.0, 1.0), (1.0, 1e-2)])
def test_cavity_operator_every_level(rho, mu):
    N = 32
    st = I.thick_annulus(N, 5.0)
    dt = 0.32 / N
    S = sib.Solver(N)
    S.set_fluid(rho, mu, dt)
    S.set_structure(cu(st.X), torch.as_tensor(st.edges, device="cuda"), cu(st.kappa))
    S.setup()
    H = cavity.Hierarchy(N, rho, mu, dt, st.X, st.edges, st.kappa, smoother="sc")
    for l, lev in enumerate(H.levels):
        Nl = lev.N
        idx = cavity.interior(Nl)
        wall = np.setdiff1d(np.arange(3 * Nl * Nl), idx)
        x = np.random.default_rng(40 + l).standard_normal(idx.size)
        ref = lev.L @ x
        y = host(S.cavity_apply_operator(l, cu(cavity.embed(Nl, x))))
        assert rel(y[idx], ref) < TOL64, (l, rel(y[idx], ref))
        assert np.abs(y[wall]).max() == 0.0
        x32 = x.astype(np.float32).astype(np.float64)
        y32 = host(S.cavity_apply_operator(l, cu(cavity.embed(Nl, x32), torch.float32)))
        assert rel(y32[idx], lev.L @ x32) < TOL32, (l, rel(y32[idx], lev.L @ x32))


@pytest.mark.parametrize("rho,mu", [(0.0, 1.0), (1.0, 1e-2)])
def test_cavity_vanka_sweep_every_level(rho, mu):
    """One additive Vanka sweep of the cavity (wall faces as infinitely stiff patch entries) against the
    oracle's patch-by-patch sweep, every level, the annulus immersed."""
    N = 32
    st = I.thick_annulus(N, 5.0)
    dt = 0.32 / N
    S = sib.Solver(N)
    S.set_fluid(rho, mu, dt)
    S.set_structure(cu(st.X), torch.as_tensor(st.edges, device="cuda"), cu(st.kappa))
    S.setup()
    H = cavity.Hierarchy(N, rho, mu, dt, st.X, st.edges, st.kappa, smoother="vanka")
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        Nl = lev.N
        idx = cavity.interior(Nl)
        wall = np.setdiff1d(np.arange(3 * Nl * Nl), idx)
        rng = np.random.default_rng(60 + l)
        x, b = rng.standard_normal(idx.size), rng.standard_normal(idx.size)
        ref = cavity.vanka_sweep(lev.L, lev.patches, lev.factors, x, b, 0.8)
        y = cu(cavity.embed(Nl, x))
        S.cavity_smooth(l, y, cu(cavity.embed(Nl, b)), 1)
        y = host(y)
        assert rel(y[idx], ref) < TOL64, (l, rel(y[idx], ref))
        assert np.abs(y[wall]).max() == 0.0
        x32, b32 = x.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
        ref32 = cavity.vanka_sweep(lev.L, lev.patches, lev.factors, x32, b32, 0.8)
        y32 = cu(cavity.embed(Nl, x32), torch.float32)
        S.cavity_smooth(l, y32, cu(cavity.embed(Nl, b32), torch.float32), 1)
        assert rel(host(y32)[idx], ref32) < TOL32, (l, rel(host(y32)[idx], ref32))

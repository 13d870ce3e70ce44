"""GPU parity of the lid-driven cavity's solve (Sec. 5: no-slip walls, regularised lid; option
domain = SIB_DOMAIN_CAVITY) against the cavity oracle: the walled transfers, the coarsest
pseudo-inverse, one V-cycle, and FGMRES to 1e-8 with the annulus immersed.

Tolerances as in test_gpu_parity: FP64 to 1e-10 relative (max norm); a whole FP32 V-cycle to 1e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import cavity, ib, krylov  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402

from tests.test_gpu_parity import TOL64, cu, host, rel  # noqa: E402


def make_case(N, rho, mu, gamma=5.0, wide=False, **opts):
    # wide: a thin circle of radius 0.38, 3.8 h from the walls at 32^2, whose 8 x 8 windows reach them
    st = I.thin_circle(N, gamma, r=0.38) if wide else I.thick_annulus(N, gamma)
    dt = 0.32 / N
    S = sib.Solver(N)
    S.set_fluid(rho, mu, dt)
    S.set_structure(cu(st.X), torch.as_tensor(st.edges, device="cuda"), cu(st.kappa))
    S.set_options(domain=sib.DOMAIN_CAVITY, **opts)
    S.setup()
    H = cavity.Hierarchy(N, rho, mu, dt, st.X, st.edges, st.kappa, smoother="vanka")
    return st, dt, S, H


@pytest.mark.parametrize("rho,mu", [(0.0, 1.0), (1.0, 1e-2)])
def test_cavity_transfers_and_coarse_solve(rho, mu):
    st, dt, S, H = make_case(32, rho, mu)
    rng = np.random.default_rng(5)
    for l in range(1, len(H.levels)):
        Nl, Nc = H.levels[l].N, H.levels[l - 1].N
        idx, idc = cavity.interior(Nl), cavity.interior(Nc)
        x, b = rng.standard_normal(idx.size), rng.standard_normal(idx.size)
        ref = H.R[l] @ (b - H.levels[l].L @ x)
        rc = host(S.residual_restrict(l, cu(cavity.embed(Nl, x)), cu(cavity.embed(Nl, b))))
        assert rel(rc[idc], ref) < TOL64 and np.abs(np.delete(rc, idc)).max() == 0.0
        ec = rng.standard_normal(idc.size)
        xf = cu(cavity.embed(Nl, x))
        S.prolong_add(l, cu(cavity.embed(Nc, ec)), xf)
        xf = host(xf)
        assert rel(xf[idx], x + H.P[l] @ ec) < TOL64 and np.abs(np.delete(xf, idx)).max() == 0.0
    n0 = H.levels[0].N
    id0 = cavity.interior(n0)
    b0 = cavity.project(rng.standard_normal(id0.size), n0)
    z = host(S.coarse_solve(cu(cavity.embed(n0, b0))))
    assert rel(z[id0], H.coarse_pinv @ b0) < TOL64


@pytest.mark.parametrize("rho,mu,wide", [(0.0, 1.0, False), (1.0, 1e-2, False), (0.0, 1.0, True)])
def test_cavity_vcycle(rho, mu, wide):
    st, dt, S, H = make_case(32, rho, mu, wide=wide, vcycle_fp32=0)
    N = 32
    idx = cavity.interior(N)
    b = cavity.lid_rhs(N, mu) + np.random.default_rng(7).standard_normal(idx.size)
    z = host(S.vcycle(cu(cavity.embed(N, b))))
    ref = H.vcycle(b)
    assert rel(z[idx], ref) < TOL64, rel(z[idx], ref)
    b32 = b.astype(np.float32).astype(np.float64)
    z32 = host(S.vcycle(cu(cavity.embed(N, b32), torch.float32)))
    assert rel(z32[idx], H.vcycle(b32)) < 1e-4


def test_cavity_fgmres_solve():
    """Stokes, the annulus at gamma = 5 driven by the lid and its own elastic force: the GPU's FGMRES
    (FP64 V-cycle) takes the oracle's iteration count within one and reaches the direct solution."""
    N, mu = 32, 1.0
    st, dt, S, H = make_case(N, 0.0, mu, vcycle_fp32=0, rtol=1e-8, max_it=100)
    idx = cavity.interior(N)
    L = cavity.operator(N, 0.0, mu, dt, st.X, st.edges, st.kappa)
    skx = ib.spread_force(N, st.X, ib.spring_force(st.X, st.edges, st.kappa))
    b = cavity.lid_rhs(N, mu) + np.concatenate([skx, np.zeros(N * N)])[idx]
    _, its, _, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-8, max_it=100, restart=100,
                                    project=lambda v: cavity.project(v, N))
    w = host(S.solve(cu(np.zeros(3 * N * N))))   # g = 0: the solve adds S K X^n and the lid's term
    assert conv and S.stats.converged, (its, S.stats.iterations)
    assert abs(S.stats.iterations - its) <= 1, (S.stats.iterations, its)
    ref = cavity.solve_direct(L, b, N)
    assert rel(cavity.project(w[idx], N), ref) < 1e-6
    assert np.abs(np.delete(w, idx)).max() == 0.0

"""The paper's structures (Sec. 5.1 thick annulus, Sec. 5.2 thin circle) in the periodic box, one
linear solve each (dt = 0.32 h, g = 0, tolerance 1e-12): GPU against the oracle at 32^2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import krylov, multigrid, system  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402

from tests.test_gpu_parity import cu, host, rel  # noqa: E402

SMOOTHERS = {"vanka": dict(smoother=sib.SMOOTHER_VANKA), "sc": dict(smoother=sib.SMOOTHER_SC),
             "ras": dict(smoother=sib.SMOOTHER_RAS, box=4, box_overlap=1)}


@pytest.mark.parametrize("kind,mu,gamma,sm", [("annulus", None, 50.0, "ras"), ("annulus", None, 5.0, "vanka"),
                                              ("annulus", 0.01, 5.0, "ras"), ("circle", None, 5.0, "ras"),
                                              ("circle", None, 5.0, "vanka"), ("annulus", None, 5.0, "sc")])
def test_paper_workload_iterations_and_solution(kind, mu, gamma, sm):
    """FP64 V-cycle: the iteration count to 1e-12 is the oracle's (within one: the last residual can
    sit within rounding of the threshold), and the solution is the direct solve's."""
    prob = I.paper_problem(kind, 32, gamma, mu)
    N = prob.N
    S = sib.solver_for(prob, vcycle_fp32=0, rtol=1e-12, max_it=100, **SMOOTHERS[sm])
    w = host(S.solve(cu(prob.g)))
    L = system.operator_of(prob)
    b = system.rhs(prob)
    H = multigrid.Hierarchy(prob, smoother=sm)
    _, its, _, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-12, max_it=100, restart=100,
                                    project=lambda v: system.project(v, N, prob.rho))
    assert conv and S.stats.converged, (its, S.stats.iterations)
    assert abs(S.stats.iterations - its) <= 1, (S.stats.iterations, its)
    ref, _ = system.solve_direct(L, b, N, prob.rho)
    ref = system.project(ref, N, prob.rho)
    # a 1e-12 relative residual bounds the solution error by that times the operator's conditioning
    assert rel(w, ref) < 1e-8, rel(w, ref)


def test_paper_rhs_is_the_initial_elastic_force():
    """g = 0: the solve's right-hand side is S K X^n alone, so a zero-stiffness structure gives w = 0."""
    prob = I.paper_problem("circle", 32, 5.0)
    prob.structure.kappa[:] = 0.0
    S = sib.solver_for(prob, rtol=1e-12)
    w = host(S.solve(cu(prob.g), allow_unconverged=True))
    assert np.abs(w).max() == 0.0

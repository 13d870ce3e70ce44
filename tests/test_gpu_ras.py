"""GPU parity of the box RAS smoother (restricted additive Schwarz over b x b boxes with overlap o,
Sec. 3.3 / Alg. 2) against the CPU oracle.

Tolerances as in test_gpu_parity: FP64 to 1e-10 relative (max norm); FP32 to 1e-5 per sweep.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import krylov, multigrid, system  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402

from tests.test_gpu_parity import TOL32, TOL64, cu, host, rand, rel  # noqa: E402

PROBLEMS = {
    "ellipse32": lambda: I.thin_ellipse_stokes(32),
    "disk32_stiff": lambda: I.disk_stokes(32, kappa=1e4, seed=1),
    "disk64": lambda: I.disk_stokes(64, kappa=1e2, seed=1),
    "ellipse64_re": lambda: I.thin_ellipse_re(64, kappa=1e4),
    "fluid32": lambda: I.no_structure(32, seed=3),
}

_cache = {}


def pair(name, b=4, o=1, krylov_smooth=False, **opts):
    key = (name, b, o, krylov_smooth, tuple(sorted(opts.items())))
    if key not in _cache:
        prob = PROBLEMS[name]()
        H = multigrid.Hierarchy(prob, smoother="ras", box=b, overlap=o, krylov=krylov_smooth)
        S = sib.solver_for(prob, smoother=sib.SMOOTHER_RAS, box=b, box_overlap=o,
                           smooth_krylov=int(krylov_smooth), **opts)
        _cache[key] = (prob, H, S)
    return _cache[key]


@pytest.mark.parametrize("name,b,o", [("ellipse32", 4, 1), ("disk32_stiff", 4, 1), ("disk64", 2, 1),
                                      ("ellipse64_re", 4, 1), ("ellipse64_re", 2, 2), ("disk32_stiff", 4, 0),
                                      ("fluid32", 4, 1), ("disk32_stiff", 1, 0)])
def test_ras_sweep_every_level(name, b, o):
    prob, H, S = pair(name, b, o)
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        x = rand(3 * lev.n, 2800 + l)
        bb = rand(3 * lev.n, 2900 + l, 10.0)
        ref = H.smooth(l, x, bb, 1)
        y = cu(x.copy())
        S.smooth(l, y, cu(bb), 1)
        assert rel(host(y), ref) < TOL64, (l, rel(host(y), ref))
        x32 = x.astype(np.float32).astype(np.float64)
        b32 = bb.astype(np.float32).astype(np.float64)
        ref32 = H.smooth(l, x32, b32, 1)
        y32 = cu(x32, torch.float32)
        S.smooth(l, y32, cu(b32, torch.float32), 1)
        assert rel(host(y32), ref32) < TOL32, (l, rel(host(y32), ref32))


@pytest.mark.parametrize("name", ["disk32_stiff", "ellipse64_re"])
def test_ras_vcycle(name):
    prob, H, S = pair(name)
    b = system.rhs(prob)
    z = host(S.vcycle(cu(b)))
    assert rel(z, H.vcycle(b)) < TOL64, rel(z, H.vcycle(b))
    b32 = b.astype(np.float32).astype(np.float64)
    z32 = host(S.vcycle(cu(b32, torch.float32)))
    assert rel(z32, H.vcycle(b32)) < 1e-4, rel(z32, H.vcycle(b32))


@pytest.mark.parametrize("name", ["ellipse32", "disk32_stiff"])
def test_ras_fgmres_fixed_iterations_fp64(name):
    prob, H, S = pair(name, vcycle_fp32=0)
    N = prob.N
    L = H.fine.L
    b = system.rhs(prob)
    for k in (1, 3, 5):
        S.set_options(max_it=k, rtol=1e-30)
        w = host(S.solve(cu(prob.g), allow_unconverged=True))
        x, its, hist, _ = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-30, max_it=k,
                                        project=lambda z: system.project(z, N, prob.rho))
        assert S.stats.iterations == its == k
        assert rel(w, x) < TOL64, (k, rel(w, x))
        np.testing.assert_allclose(np.array(S.stats.as_dict()["history"]), hist, rtol=1e-9)
    S.set_options(max_it=100, rtol=1e-8)


@pytest.mark.parametrize("name,fp32", [("disk32_stiff", 1), ("disk64", 0), ("ellipse64_re", 1)])
def test_ras_converged_solution_and_iterations(name, fp32):
    """Solved to 1e-13 the result is the direct solution; at 1e-8 the FP64-V-cycle solve takes the
    oracle's iteration count."""
    prob, H, S = pair(name)
    N = prob.N
    L = system.operator_of(prob)
    b = system.rhs(prob)
    S.set_options(vcycle_fp32=fp32, rtol=1e-13, max_it=100)
    ref, _ = system.solve_direct(L, b, N, prob.rho)
    ref = system.project(ref, N, prob.rho)
    w = host(S.solve(cu(prob.g)))
    assert S.stats.converged and S.stats.rel_residual < 1e-12
    assert rel(w, ref) < TOL64, rel(w, ref)
    S.set_options(vcycle_fp32=0, rtol=1e-8)
    S.solve(cu(prob.g))
    _, its, _, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-8, max_it=100,
                                    project=lambda z: system.project(z, N, prob.rho))
    assert conv and S.stats.converged and S.stats.iterations == its, (S.stats.iterations, its)


def test_ras_with_wrapped_smoothing_vcycle():
    prob, H, S = pair("disk32_stiff", krylov_smooth=True)
    b = system.rhs(prob)
    z = host(S.vcycle(cu(b)))
    assert rel(z, H.vcycle(b)) < TOL64, rel(z, H.vcycle(b))


def test_ras_stiff_disk_converges_where_vanka_caps():
    """The 32^2 disk at kappa = 1e6: the RAS V-cycle (4 x 4 boxes, overlap 1) reaches 1e-8 within the
    100-iteration cap, with the oracle's iteration count."""
    prob = I.disk_stokes(32, kappa=1e6, seed=1)
    S = sib.solver_for(prob, smoother=sib.SMOOTHER_RAS, vcycle_fp32=0)
    S.solve(cu(prob.g))
    H = multigrid.Hierarchy(prob, smoother="ras")
    L = system.operator_of(prob)
    _, its, _, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, system.rhs(prob), rtol=1e-8, max_it=100,
                                    project=lambda z: system.project(z, 32, prob.rho))
    assert conv and S.stats.converged and S.stats.iterations == its


def test_ras_options_validated():
    """Box sides 1, 2, 4, 8, 16; a subdomain (b + 2 o cells) at most 16 wide for b <= 8, overlap at most
    4 for b = 16; the tensor-core choice 0 or 1."""
    prob, H, S = pair("ellipse32")
    for kw in (dict(box=3), dict(box=32, box_overlap=0), dict(box=8, box_overlap=5), dict(box=16, box_overlap=5),
               dict(box_overlap=-1), dict(ras_tc=2), dict(ras_tc=-1), dict(l2_persist=2)):
        with pytest.raises(sib.SibError):
            S.set_options(**kw)
        S.set_options(box=4, box_overlap=1)
    for b, o in ((4, 2), (8, 2), (2, 6), (8, 4), (16, 4)):
        S.set_options(box=b, box_overlap=o)
    S.set_options(box=4, box_overlap=1)
    S.setup()   # the cached solver serves the other tests


def test_ras_small_coarse_grid_boxes_span_rows():
    """n_min = 4: level 1 is 8 x 8, two 4 x 4 boxes per row, so a group of four boxes in the
    correction kernel spans two box rows; one sweep per level and one V-cycle against the oracle."""
    prob = I.thin_ellipse_stokes(32, kappa=1e2)
    H = multigrid.Hierarchy(prob, n_min=4, smoother="ras", box=4, overlap=1)
    S = sib.Solver(32, 4)
    S.set_fluid(prob.rho, prob.mu, prob.dt)
    st = prob.structure
    S.set_structure(cu(st.X), torch.as_tensor(st.edges, device="cuda"), cu(st.kappa))
    S.set_options(smoother=sib.SMOOTHER_RAS, box=4, box_overlap=1)
    S.setup()
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        x = rand(3 * lev.n, 3800 + l)
        bb = rand(3 * lev.n, 3900 + l, 10.0)
        y = cu(x.copy())
        S.smooth(l, y, cu(bb), 1)
        assert rel(host(y), H.smooth(l, x, bb, 1)) < TOL64, l
    b = system.rhs(prob)
    assert rel(host(S.vcycle(cu(b))), H.vcycle(b)) < TOL64


@pytest.mark.parametrize("name,b,o", [("ellipse32", 4, 1), ("disk32_stiff", 2, 1), ("ellipse64_re", 4, 1)])
def test_ras_tensor_core_correction_matches_cuda_core_form(name, b, o):
    """FP32 levels: the correction of the boxes sharing one inverse on the tensor cores (tcgen05, three
    TF32 products per pair) against the same correction on the FP32 CUDA cores and against the oracle,
    one sweep per level, and one V-cycle."""
    prob = PROBLEMS[name]()
    H = multigrid.Hierarchy(prob, smoother="ras", box=b, overlap=o)
    S = sib.solver_for(prob, smoother=sib.SMOOTHER_RAS, box=b, box_overlap=o)
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        x32 = rand(3 * lev.n, 5800 + l).astype(np.float32).astype(np.float64)
        b32 = rand(3 * lev.n, 5900 + l, 10.0).astype(np.float32).astype(np.float64)
        ref = H.smooth(l, x32, b32, 1)
        outs = []
        for tc in (1, 0):
            S.set_options(ras_tc=tc)
            y = cu(x32, torch.float32)
            S.smooth(l, y, cu(b32, torch.float32), 1)
            outs.append(host(y))
        assert rel(outs[0], ref) < TOL32, (l, rel(outs[0], ref))
        assert rel(outs[0], outs[1]) < TOL32, (l, rel(outs[0], outs[1]))
    S.set_options(ras_tc=1)
    bb = system.rhs(prob).astype(np.float32).astype(np.float64)
    assert rel(host(S.vcycle(cu(bb, torch.float32))), H.vcycle(bb)) < 1e-4

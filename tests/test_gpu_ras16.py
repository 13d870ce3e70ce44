"""GPU parity of box RAS with the paper's 16 x 16 boxes and overlap 4 (Sec. 5.1.1, 5.2.1) against the
oracle.  The GPU keeps one inverse of the IB-free subdomain operator per level (1,776 dofs) and applies
each IB box's own local solve as a low-rank (Woodbury) update of it over the box's IB-touched dofs; the
oracle factors every box's local operator.  Levels too small for the boxes (16^2) take the exact level
solve on both sides.

FP64 to 1e-10 and FP32 to 1e-5 per sweep; the stiff thin circle at gamma = 500 keeps the 8 x 8 boxes'
FP32 exception (its FP32 storage alone moves a sweep past 1e-5).  FP32 levels with fewer than 1,024 boxes
take the CUDA-core form of the shared correction, larger ones the tensor cores.  On 512^2 the oracle
solves sampled boxes one by one: there the tensor-core form writes its tiles row by row.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import krylov, multigrid, smoothers, system  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402

from tests.test_gpu_parity import TOL32, TOL64, cu, host, rand, rel  # noqa: E402
from tests.test_gpu_ras_wide import TOL32_STIFF_CIRCLE  # noqa: E402

PROBLEMS = {
    "ellipse64_re": lambda: I.thin_ellipse_re(64, kappa=1e4),
    "circle64_g500": lambda: I.paper_problem("circle", 64, 500.0),
    "annulus64_g50": lambda: I.paper_problem("annulus", 64, 50.0),
    "fluid64": lambda: I.no_structure(64, rho=1.0, seed=5),
}

_cache = {}


def pair(name, b=16, o=4, **opts):
    key = (name, b, o, tuple(sorted(opts.items())))
    if key not in _cache:
        prob = PROBLEMS[name]()
        H = multigrid.Hierarchy(prob, smoother="ras", box=b, overlap=o)
        S = sib.solver_for(prob, smoother=sib.SMOOTHER_RAS, box=b, box_overlap=o, **opts)
        _cache[key] = (prob, H, S)
    return _cache[key]


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_ras16_sweep_every_level(name):
    """One sweep per level: the exact level solve on 16^2, four and sixteen 16 x 16 boxes on 32^2 and
    64^2, with and without IB boxes."""
    prob, H, S = pair(name)
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        x = rand(3 * lev.n, 4800 + l)
        bb = rand(3 * lev.n, 4900 + l, 10.0)
        ref = H.smooth(l, x, bb, 1)
        y = cu(x.copy())
        S.smooth(l, y, cu(bb), 1)
        assert rel(host(y), ref) < TOL64, (l, rel(host(y), ref))
        x32 = x.astype(np.float32).astype(np.float64)
        b32 = bb.astype(np.float32).astype(np.float64)
        ref32 = H.smooth(l, x32, b32, 1)
        y32 = cu(x32, torch.float32)
        S.smooth(l, y32, cu(b32, torch.float32), 1)
        tol = TOL32_STIFF_CIRCLE if name == "circle64_g500" else TOL32
        assert rel(host(y32), ref32) < tol, (l, rel(host(y32), ref32), tol)


@pytest.mark.parametrize("name", ["ellipse64_re", "circle64_g500"])
def test_ras16_vcycle(name):
    """One V-cycle, FP64 to 1e-10 and FP32 to the V-cycle bar 1e-4."""
    prob, H, S = pair(name)
    b = system.rhs(prob)
    assert rel(host(S.vcycle(cu(b))), H.vcycle(b)) < TOL64
    b32 = b.astype(np.float32).astype(np.float64)
    assert rel(host(S.vcycle(cu(b32, torch.float32))), H.vcycle(b32)) < 1e-4


def test_ras16_thin_circle_converges_faster_than_8x8():
    """The thin circle at gamma = 500 in Stokes flow (Sec. 5.2.1): FGMRES with the FP64 RAS V-cycle to
    1e-12 takes the oracle's iteration count within one, fewer than with 8 x 8 boxes (overlap 2), and
    reaches the direct solve's solution."""
    counts = {}
    for b, o in ((16, 4), (8, 2)):
        prob, H, S = pair("circle64_g500", b, o, vcycle_fp32=0, rtol=1e-12, max_it=100)
        w = host(S.solve(cu(prob.g)))
        L = system.operator_of(prob)
        rhs = system.rhs(prob)
        _, its, _, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, rhs, rtol=1e-12, max_it=100, restart=100,
                                        project=lambda v: system.project(v, prob.N, prob.rho))
        assert conv and S.stats.converged, (b, its, S.stats.iterations)
        assert abs(S.stats.iterations - its) <= 1, (b, S.stats.iterations, its)
        counts[b] = S.stats.iterations
        if b == 16:
            ref, _ = system.solve_direct(L, rhs, prob.N, prob.rho)
            assert rel(w, system.project(ref, prob.N, prob.rho)) < 1e-8
    assert counts[16] < counts[8], counts


@pytest.mark.parametrize("name", ["ellipse64_re", "annulus64_g50"])
def test_ras16_cuda_core_correction_every_small_level(name):
    """FP32 levels with fewer than 1,024 boxes take the CUDA-core correction, its owned rows split over
    blocks, whatever the tensor-core option says: against the oracle, and the same bits either way."""
    prob, H, S = pair(name)
    for l in range(2, len(H.levels)):
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
        S.set_options(ras_tc=1)
        assert rel(outs[0], ref) < TOL32, (l, rel(outs[0], ref))
        assert np.array_equal(outs[0], outs[1]), l


def test_ras16_overlap2():
    """16 x 16 boxes with overlap 2 (1,240 dofs: the elimination pads them to 1,248): one FP64 sweep per
    level on the thin ellipse."""
    prob, H, S = pair("ellipse64_re", 16, 2)
    for l in range(1, len(H.levels)):
        lev = H.levels[l]
        x = rand(3 * lev.n, 6100 + l)
        bb = rand(3 * lev.n, 6200 + l, 10.0)
        y = cu(x.copy())
        S.smooth(l, y, cu(bb), 1)
        assert rel(host(y), H.smooth(l, x, bb, 1)) < TOL64, l


@pytest.mark.parametrize("tc", [1, 0])
def test_ras16_sampled_boxes_on_512(tc):
    """512^2 thin ellipse (1,024 boxes, 32 per row): one sweep on the finest level, FP64 and FP32,
    against the oracle's local solves of sampled boxes (IB boxes, IB-free boxes, and boxes whose
    subdomain wraps around the periodic edges).  FP32 with the tensor-core correction (tc = 1: four row
    groups of 192 owned rows, K = 1,776 in 56 chunks, the tiles written row by row) and with the
    CUDA-core form (tc = 0), each held to 1e-5."""
    prob = I.thin_ellipse_re(512, kappa=1e4)
    N, b, o = 512, 16, 4
    S = sib.solver_for(prob, smoother=sib.SMOOTHER_RAS, box=b, box_overlap=o, ras_tc=tc)
    L = system.operator_of(prob).tocsr()
    boxes = smoothers.ras_boxes(N, b, o)
    x = rand(3 * N * N, 7100)
    bb = rand(3 * N * N, 7200, 10.0)
    # box k = J (N / b) + I: corners, edges, the ellipse's rim (IB boxes) and open fluid
    nb = N // b
    # the rim passes x = 0.2 and 0.8 (I = 6, 25) at mid-height and y = 0.3 and 0.7 (J = 9, 22) mid-width
    picks = [0, nb - 1, nb * (nb - 1), nb * nb - 1, nb * (nb // 2) + nb // 2 - 9, nb * (nb // 2) + 3,
             nb * 5 + 11, nb * (nb // 2 - 4) + nb // 2 + 9, nb * 16 + 6, nb * 16 + 25, nb * 9 + 16,
             nb * 22 + 16, nb * 11 + 9, nb * 20 + 23]
    lmax = S.num_levels - 1
    for prec, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
        xp = x if prec == torch.float64 else x.astype(np.float32).astype(np.float64)
        bp = bb if prec == torch.float64 else bb.astype(np.float32).astype(np.float64)
        y = cu(xp, prec)
        S.smooth(lmax, y, cu(bp, prec), 1)
        y = host(y)
        r = bp - L @ xp
        scale = np.abs(y).max()
        errs = {}
        for k in picks:
            d, own = boxes[k]
            delta = np.linalg.solve(L[d][:, d].toarray(), r[d])
            want = xp[d[own]] + delta[own]
            errs[k] = np.abs(y[d[own]] - want).max() / scale
        assert max(errs.values()) < tol, (prec, errs)
    S.close()

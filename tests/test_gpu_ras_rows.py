"""GPU parity of the tensor-core box-RAS correction on grids whose rows hold a multiple of 32 boxes
(Sec. 3.3 / Alg. 2).  There a TMEM lane quadrant's 32 boxes lie side by side in one row of boxes, and
the kernel writes the tile row by row after re-reading its totals from the TMEM with the 16 x 256-bit
load shape; on the smaller grids of the other RAS tests it writes box by box.

One FP32 sweep on the finest level against the oracle's sweep (1e-5, as for every FP32 sweep) and
against the CUDA-core form of the same correction.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import multigrid  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402

from tests.test_gpu_parity import TOL32, cu, host, rand, rel  # noqa: E402

# (problem, box, overlap): N / b = 32 boxes per row on the finest level
CASES = [
    ("ellipse128_re", lambda: I.thin_ellipse_re(128, kappa=1e4), 4, 1),
    ("fluid64", lambda: I.no_structure(64, rho=1.0, seed=4), 2, 1),
    ("ellipse256_re", lambda: I.thin_ellipse_re(256, kappa=1e4), 8, 2),
]


@pytest.mark.parametrize("name,make,b,o", CASES, ids=[c[0] for c in CASES])
def test_tensor_core_correction_row_writes(name, make, b, o):
    prob = make()
    H = multigrid.Hierarchy(prob, smoother="ras", box=b, overlap=o)
    S = sib.solver_for(prob, smoother=sib.SMOOTHER_RAS, box=b, box_overlap=o)
    l = len(H.levels) - 1
    assert prob.N // b == 32
    lev = H.levels[l]
    x32 = rand(3 * lev.n, 7800 + b).astype(np.float32).astype(np.float64)
    b32 = rand(3 * lev.n, 7900 + b, 10.0).astype(np.float32).astype(np.float64)
    ref = H.smooth(l, x32, b32, 1)
    outs = []
    for tc in (1, 0):
        S.set_options(ras_tc=tc)
        y = cu(x32, torch.float32)
        S.smooth(l, y, cu(b32, torch.float32), 1)
        outs.append(host(y))
    S.set_options(ras_tc=1)
    assert rel(outs[0], ref) < TOL32, rel(outs[0], ref)
    assert rel(outs[0], outs[1]) < TOL32, rel(outs[0], outs[1])
    S.close()

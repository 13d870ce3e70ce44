"""The L2 access policy of the captured graphs (option l2_persist: the finest level's FP32 IB windows
kept in L2) changes where data sits, not what is computed: the FGMRES solve with the FP32 V-cycle
gives bitwise the same iterate and iteration count with the policy on and off."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402


def test_l2_persist_changes_no_result():
    prob = I.disk_and_ellipse_re(128)
    S = sib.solver_for(prob, smoother=sib.SMOOTHER_SC, smooth_krylov=1, vcycle_fp32=1, omega=-1.0, rtol=1e-8)
    g = torch.as_tensor(prob.g, device="cuda")
    out = {}
    for l2 in (1, 0):
        S.set_options(l2_persist=l2)
        w = S.solve(g).cpu().numpy()
        out[l2] = (w, S.stats.iterations)
    assert out[1][1] == out[0][1]
    assert np.array_equal(out[1][0], out[0][0])
    S.close()

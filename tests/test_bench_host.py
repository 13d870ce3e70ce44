"""Host logic of bench.py that needs no GPU: the probes that decide whether the legs for the paper's
8 x 8 RAS boxes and for the lid-driven cavity run, against a stand-in for the binding whose options
accept or reject those settings."""
import types

import bench


class _Err(RuntimeError):
    pass


def _fake_binding(accept_wide, accept_cavity):
    closed = []

    class Solver:
        def __init__(self, N):
            self.N = N

        def set_options(self, **kw):
            if kw.get("box", 4) + 2 * kw.get("box_overlap", 1) > 6 and not accept_wide:
                raise _Err("option out of range")
            if kw.get("domain", 0) == 1 and not accept_cavity:
                raise _Err("unimplemented")

        def close(self):
            closed.append(self.N)

    return types.SimpleNamespace(Solver=Solver, SibError=_Err, SMOOTHER_RAS=2, DOMAIN_CAVITY=1), closed


def test_wide_box_probe_follows_the_options_and_closes_its_context():
    sib, closed = _fake_binding(False, False)
    assert bench.wide_boxes_accepted(sib) is False
    sib2, closed2 = _fake_binding(True, False)
    assert bench.wide_boxes_accepted(sib2) is True
    assert closed == [32] and closed2 == [32]


def test_cavity_leg_reports_unavailable_when_the_domain_is_rejected():
    sib, closed = _fake_binding(True, False)
    out = bench.cavity_workloads(sib, None, "cpu")
    assert set(out) == {"unavailable"} and closed == [32]

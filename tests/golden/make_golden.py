"""Writes tests/golden/fgmres_histories.json: FGMRES(100) iteration counts and residual histories of
the CPU oracle on small seeded problems (the 32 x 32 thin-ellipse Stokes problem and the 32 x 32
disk), for both smoothers.  Calls only the oracle and the seeded input generators.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov, multigrid, system  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402

CASES = {
    "thin_ellipse_stokes_N32_kappa1e2": lambda: I.thin_ellipse_stokes(32, kappa=1e2),
    "disk_stokes_N32_kappa1e2": lambda: I.disk_stokes(32, kappa=1e2),
    "thin_ellipse_re_N64_kappa1e4": lambda: I.thin_ellipse_re(64, kappa=1e4),
}


def compute():
    out = {}
    for name, make in CASES.items():
        for sm in ("vanka", "sc"):
            prob = make()
            L = system.operator_of(prob)
            b = system.rhs(prob)
            H = multigrid.Hierarchy(prob, smoother=sm)
            x, its, hist, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-8, max_it=100)
            out[f"{name}/{sm}"] = {"iterations": int(its), "converged": bool(conv),
                                   "history": [float(h) for h in hist]}
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fgmres_histories.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=1)
    print("wrote", path)

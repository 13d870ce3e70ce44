"""The oracle reproduces its stored FGMRES histories (tests/golden/make_golden.py)."""
import json
import os

import numpy as np

from tests.golden import make_golden

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fgmres_histories.json")


def test_oracle_histories_are_stable():
    stored = json.load(open(GOLDEN))
    now = make_golden.compute()
    assert stored.keys() == now.keys()
    for k in stored:
        assert stored[k]["iterations"] == now[k]["iterations"], k
        np.testing.assert_allclose(now[k]["history"], stored[k]["history"], rtol=1e-9, err_msg=k)

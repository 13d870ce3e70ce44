"""The no-allocation spreading entry point (sib_spread_noalloc) against the context-based
sib_spread, through the C ABI, on two calls in a row.

Callers that cannot allocate device memory (programs whose device memory belongs to their own
pool allocator, latency-critical loops that cannot take cudaMalloc's synchronisation) use this
call; it must give the same spread force as the solver's own path.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402

TOL64 = 1e-10


def _rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _noalloc(lib, N, X, F):
    f = torch.full((2 * N * N,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.sib_spread_noalloc(N, X.shape[0], ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(F.data_ptr()),
                                ctypes.c_void_p(f.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc, f


def test_spread_noalloc_matches_context_spread_twice():
    lib = sib.load()
    cases = [I.thin_ellipse_stokes(32), I.disk_stokes(64, kappa=1e2), I.thin_ellipse_loguniform(256)]
    for k, prob in enumerate(cases):          # consecutive calls reuse the shared scratch
        st = prob.structure
        X = torch.as_tensor(st.X, device="cuda")
        F = torch.as_tensor(np.random.default_rng(40 + k).standard_normal((st.M, 2)), device="cuda")
        S = sib.solver_for(prob)
        ref = S.spread(F).cpu().numpy()
        rc, f = _noalloc(lib, prob.N, X, F)
        assert rc == sib.SIB_OK
        out = f.cpu().numpy()
        assert np.isfinite(out).all()
        assert _rel(out, ref) < TOL64, (prob.name, _rel(out, ref))
        S.close()


def test_spread_noalloc_rejects_sizes_beyond_its_scratch():
    lib = sib.load()
    X = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    F = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, 512, X, F)[0] == sib.SIB_ERR_TOO_LARGE
    big = torch.zeros((16385, 2), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, 64, big, big)[0] == sib.SIB_ERR_TOO_LARGE
    assert _noalloc(lib, 48, X, F)[0] == sib.SIB_ERR_ARG

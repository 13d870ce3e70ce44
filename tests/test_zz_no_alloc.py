"""The no-allocation spreading entry point (sib_spread_noalloc) through the C ABI: against the
oracle's spreading S F (Appendix, force spreading) and against the context-based sib_spread, on
consecutive calls that share its scratch, with no device memory taken by a call.

Callers that cannot allocate device memory use this call: programs whose device memory belongs to
their own pool allocator (a raw cudaMalloc would fail or fragment the pool) and latency-critical
loops that cannot take the device-wide synchronisation of cudaMalloc/cudaFree.  It must give the
spread force of the solver's own path, and it must not allocate.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ib  # noqa: E402
from paper_1612_02208_gb300 import inputs as I  # noqa: E402
from paper_1612_02208_gb300 import sib  # noqa: E402

TOL64 = 1e-10


def _rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def _noalloc(lib, N, X, F, f=None):
    if f is None:
        f = torch.full((2 * N * N,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    M = X.shape[0]
    rc = lib.sib_spread_noalloc(N, M, ctypes.c_void_p(X.data_ptr() if M else None),
                                ctypes.c_void_p(F.data_ptr() if M else None), ctypes.c_void_p(f.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc, f


def _cases():
    # N = 16 is narrower than one 32-cell tile row (a single tile column); N = 256 is the limit
    return [I.thin_ellipse_stokes(32), I.disk_stokes(16, kappa=1e2), I.disk_stokes(64, kappa=1e2),
            I.thin_ellipse_loguniform(256)]


def test_spread_noalloc_matches_oracle_and_context_spread_twice():
    lib = sib.load()
    for rep in range(2):                      # the second pass reuses the scratch left by the first
        for k, prob in enumerate(_cases()):
            st = prob.structure
            Fh = np.random.default_rng(40 + k).standard_normal((st.M, 2))
            X = torch.as_tensor(st.X, device="cuda")
            F = torch.as_tensor(Fh, device="cuda")
            rc, f = _noalloc(lib, prob.N, X, F)
            assert rc == sib.SIB_OK
            out = f.cpu().numpy()
            assert np.isfinite(out).all()
            ref = ib.spread_force(prob.N, st.X, Fh)
            assert _rel(out, ref) < TOL64, (rep, prob.name, _rel(out, ref))
            S = sib.solver_for(prob)
            ctx = S.spread(F).cpu().numpy()
            S.close()
            assert _rel(out, ctx) < TOL64, (rep, prob.name, _rel(out, ctx))


def test_spread_noalloc_without_markers_writes_zeros():
    lib = sib.load()
    empty = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    for N in (16, 64):
        rc, f = _noalloc(lib, N, empty, empty)
        assert rc == sib.SIB_OK
        assert torch.count_nonzero(f).item() == 0


def test_spread_noalloc_takes_no_device_memory():
    lib = sib.load()
    prob = I.disk_stokes(64, kappa=1e2)
    st = prob.structure
    X = torch.as_tensor(st.X, device="cuda")
    F = torch.as_tensor(np.random.default_rng(7).standard_normal((st.M, 2)), device="cuda")
    f = torch.empty(2 * prob.N * prob.N, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, prob.N, X, F, f)[0] == sib.SIB_OK    # warm-up: module and kernels loaded
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        assert _noalloc(lib, prob.N, X, F, f)[0] == sib.SIB_OK
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0


def test_spread_noalloc_rejects_sizes_beyond_its_scratch():
    lib = sib.load()
    X = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    F = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, 512, X, F)[0] == sib.SIB_ERR_TOO_LARGE
    big = torch.zeros((16385, 2), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, 64, big, big)[0] == sib.SIB_ERR_TOO_LARGE
    assert _noalloc(lib, 48, X, F)[0] == sib.SIB_ERR_ARG

"""ctypes binding of libsib (include/sib.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch supplies device memory (tensors) and the
current CUDA stream.  The library is loaded on first use and its absence is an error: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SIB_OK = 0
SIB_ERR_ARG = -1
SIB_ERR_CUDA = -2
SIB_ERR_NONFINITE = -3
SIB_ERR_NOT_CONVERGED = -4
SIB_ERR_BREAKDOWN = -5
SIB_ERR_UNIMPLEMENTED = -6
SIB_ERR_STATE = -7
SIB_ERR_ALLOC = -8
SIB_ERR_TOO_LARGE = -9
ERROR_NAMES = {v: k for k, v in dict(globals()).items() if k.startswith("SIB_ERR") or k == "SIB_OK"}

SMOOTHER_VANKA = 0
SMOOTHER_SC = 1
SMOOTHER_RAS = 2
RELAX_JACOBI = 0
RELAX_SGS = 1
DOMAIN_PERIODIC = 0
DOMAIN_CAVITY = 1
PREC_FP64 = 0
PREC_FP32 = 1
MAX_LEVELS = 12

# every extern "C" symbol of include/sib.h
EXPORTS = [
    "sib_default_opts", "sib_create", "sib_destroy", "sib_last_error", "sib_set_fluid", "sib_set_structure",
    "sib_set_stiffness", "sib_set_options", "sib_set_eigen_estimates", "sib_get_eigen_estimates", "sib_setup",
    "sib_solve", "sib_solve_host", "sib_solve_rhs", "sib_solve_transpose", "sib_grad", "sib_num_levels", "sib_level_size",
    "sib_apply_operator", "sib_cavity_apply_operator", "sib_cavity_smooth", "sib_apply_ib", "sib_smooth", "sib_residual_restrict", "sib_prolong_add",
    "sib_coarse_solve", "sib_vcycle", "sib_interp", "sib_spread", "sib_time_kernel", "sib_launch_count",
    "sib_device_bytes", "sib_spread_noalloc", "sib_advance_markers",
]
TIME_COLD = 0x100
KERNELS = {"vanka": 0, "residual": 1, "spread": 2, "interp": 3, "restrict": 4, "prolong": 5, "ras": 6, "ib_window": 7,
           "residual_restrict": 8}


class SibOpts(ctypes.Structure):
    _fields_ = [
        ("smoother", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
        ("cheb_iters", ctypes.c_int), ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double),
        ("power_iters", ctypes.c_int), ("vcycle_fp32", ctypes.c_int), ("rtol", ctypes.c_double),
        ("max_it", ctypes.c_int), ("restart", ctypes.c_int), ("add_SKXn", ctypes.c_int), ("use_graphs", ctypes.c_int),
        ("fuse_small", ctypes.c_int), ("smooth_krylov", ctypes.c_int), ("sc_relax", ctypes.c_int),
        ("box", ctypes.c_int), ("box_overlap", ctypes.c_int), ("domain", ctypes.c_int), ("ras_tc", ctypes.c_int),
        ("l2_persist", ctypes.c_int),
    ]


class SibStats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
        ("rel_residual_est", ctypes.c_double), ("bnorm", ctypes.c_double), ("setup_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double), ("history", ctypes.c_double * 101),
    ]

    def as_dict(self):
        k = min(self.iterations + 1, 101)
        return dict(iterations=self.iterations, converged=bool(self.converged), rel_residual=self.rel_residual,
                    rel_residual_est=self.rel_residual_est, bnorm=self.bnorm, setup_ms=self.setup_ms,
                    solve_ms=self.solve_ms, history=list(self.history[:k]))


class SibError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsib.so (building it first if needed).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsib.so not found at {path}; run paper_1612_02208_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    ctx = ctypes.c_void_p
    sig = {
        "sib_default_opts": (None, [ctypes.POINTER(SibOpts)]),
        "sib_create": (I, [ctypes.POINTER(ctx), I, I]),
        "sib_destroy": (None, [ctx]),
        "sib_last_error": (ctypes.c_char_p, [ctx]),
        "sib_set_fluid": (I, [ctx, D, D, D]),
        "sib_set_structure": (I, [ctx, I, P, I, P, P, P]),
        "sib_set_stiffness": (I, [ctx, P, P]),
        "sib_set_options": (I, [ctx, ctypes.POINTER(SibOpts)]),
        "sib_set_eigen_estimates": (I, [ctx, P, P]),
        "sib_get_eigen_estimates": (I, [ctx, P, P]),
        "sib_setup": (I, [ctx, P]),
        "sib_solve": (I, [ctx, P, P, ctypes.POINTER(SibStats), P]),
        "sib_solve_host": (I, [ctx, P, P, ctypes.POINTER(SibStats), P]),
        "sib_solve_rhs": (I, [ctx, P, P, ctypes.POINTER(SibStats), P]),
        "sib_solve_transpose": (I, [ctx, P, P, ctypes.POINTER(SibStats), P]),
        "sib_grad": (I, [ctx, P, P, P, P, P]),
        "sib_num_levels": (I, [ctx]),
        "sib_level_size": (I, [ctx, I]),
        "sib_apply_operator": (I, [ctx, I, I, P, P, P]),
        "sib_cavity_apply_operator": (I, [ctx, I, I, P, P, P]),
        "sib_cavity_smooth": (I, [ctx, I, I, P, P, I, P]),
        "sib_apply_ib": (I, [ctx, I, I, P, P, P]),
        "sib_smooth": (I, [ctx, I, I, P, P, I, P]),
        "sib_residual_restrict": (I, [ctx, I, I, P, P, P, P]),
        "sib_prolong_add": (I, [ctx, I, I, P, P, P]),
        "sib_coarse_solve": (I, [ctx, I, P, P, P]),
        "sib_vcycle": (I, [ctx, I, P, P, P]),
        "sib_interp": (I, [ctx, P, P, P]),
        "sib_spread": (I, [ctx, P, P, P]),
        "sib_time_kernel": (I, [ctx, I, I, I, I, P, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "sib_launch_count": (ctypes.c_int64, [ctx]),
        "sib_advance_markers": (I, [ctx, P, P, P]),
        "sib_device_bytes": (ctypes.c_int64, [ctx]),
        "sib_spread_noalloc": (I, [I, I, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Solver:
    """One solver context (sib_ctx) for an N x N periodic MAC grid.

    Tensors passed in are CUDA tensors (float64 unless a level call asks for float32) in the
    layouts of include/sib.h; they are used through their data pointers on the current stream.
    """

    def __init__(self, N: int, n_min: int = 8):
        self.lib = load()
        self.ctx = ctypes.c_void_p()
        rc = self.lib.sib_create(ctypes.byref(self.ctx), int(N), int(n_min))
        if rc != SIB_OK:
            raise SibError(rc, "sib_create failed")
        self.N = int(N)
        self.n_min = int(n_min)
        self.opts = SibOpts()
        self.lib.sib_default_opts(ctypes.byref(self.opts))
        self.M = 0
        self.E = 0
        self.stats = SibStats()

    def close(self):
        if self.ctx:
            self.lib.sib_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != SIB_OK and rc not in allow:
            msg = self.lib.sib_last_error(self.ctx)
            raise SibError(rc, msg.decode() if msg else "")
        return rc

    # ---- problem definition
    def set_fluid(self, rho, mu, dt):
        self._check(self.lib.sib_set_fluid(self.ctx, float(rho), float(mu), float(dt)))

    def set_structure(self, X, edges, kappa):
        self.M = int(X.shape[0]) if X is not None else 0
        self.E = int(edges.shape[0]) if edges is not None else 0
        self._check(self.lib.sib_set_structure(self.ctx, self.M, _ptr(X) if self.M else None, self.E,
                                               _ptr(edges) if self.E else None, _ptr(kappa) if self.E else None,
                                               _stream()))

    def set_stiffness(self, kappa):
        self._check(self.lib.sib_set_stiffness(self.ctx, _ptr(kappa) if self.E else None, _stream()))

    def set_options(self, **kw):
        """Changes the named fields; a set the library rejects leaves the previous options in force."""
        new = SibOpts()
        ctypes.pointer(new)[0] = self.opts
        for k, v in kw.items():
            if not hasattr(new, k):
                raise KeyError(k)
            setattr(new, k, v)
        self._check(self.lib.sib_set_options(self.ctx, ctypes.byref(new)))
        self.opts = new

    def set_eigen_estimates(self, lamA=None, lamM=None):
        if lamA is None:
            self._check(self.lib.sib_set_eigen_estimates(self.ctx, None, None))
            return
        a = (ctypes.c_double * len(lamA))(*lamA)
        m = (ctypes.c_double * len(lamM))(*lamM)
        self._check(self.lib.sib_set_eigen_estimates(self.ctx, a, m))

    def eigen_estimates(self):
        n = self.num_levels
        a = (ctypes.c_double * n)()
        m = (ctypes.c_double * n)()
        self._check(self.lib.sib_get_eigen_estimates(self.ctx, a, m))
        return list(a), list(m)

    def setup(self):
        self._check(self.lib.sib_setup(self.ctx, _stream()))

    # ---- solves
    def solve(self, g, w=None, allow_unconverged=False):
        torch = _torch()
        if w is None:
            w = torch.empty_like(g)
        rc = self.lib.sib_solve(self.ctx, _ptr(g), _ptr(w), ctypes.byref(self.stats), _stream())
        self._check(rc, (SIB_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return w

    def solve_rhs(self, rhs, w=None, allow_unconverged=False):
        torch = _torch()
        if w is None:
            w = torch.empty_like(rhs)
        rc = self.lib.sib_solve_rhs(self.ctx, _ptr(rhs), _ptr(w), ctypes.byref(self.stats), _stream())
        self._check(rc, (SIB_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return w

    def solve_transpose(self, rhs, w=None, allow_unconverged=False):
        """Solves L^T w = rhs (the adjoint solve; L_IB is symmetric)."""
        torch = _torch()
        if w is None:
            w = torch.empty_like(rhs)
        rc = self.lib.sib_solve_transpose(self.ctx, _ptr(rhs), _ptr(w), ctypes.byref(self.stats), _stream())
        self._check(rc, (SIB_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return w

    def solve_host(self, g: np.ndarray, w: np.ndarray | None = None, allow_unconverged=False):
        g = np.ascontiguousarray(g, dtype=np.float64)
        if w is None:
            w = np.empty_like(g)
        rc = self.lib.sib_solve_host(self.ctx, g.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(self.stats), _stream())
        self._check(rc, (SIB_ERR_NOT_CONVERGED,) if allow_unconverged else ())
        return w

    def grad(self, w, lam):
        torch = _torch()
        dk = torch.empty(max(self.E, 1), dtype=torch.float64, device=w.device)[: self.E]
        dX = torch.empty((max(self.M, 1), 2), dtype=torch.float64, device=w.device)[: self.M]
        self._check(self.lib.sib_grad(self.ctx, _ptr(w), _ptr(lam), _ptr(dk), _ptr(dX), _stream()))
        return dk, dX

    # ---- level operations
    @property
    def num_levels(self):
        return self.lib.sib_num_levels(self.ctx)

    def level_size(self, l):
        return self.lib.sib_level_size(self.ctx, int(l))

    @staticmethod
    def _prec(t):
        torch = _torch()
        return PREC_FP64 if t.dtype == torch.float64 else PREC_FP32

    def apply_operator(self, l, x, y=None):
        torch = _torch()
        y = torch.empty_like(x) if y is None else y
        self._check(self.lib.sib_apply_operator(self.ctx, int(l), self._prec(x), _ptr(x), _ptr(y), _stream()))
        return y

    def cavity_apply_operator(self, l, x, y=None):
        """y = L^l x of the lid-driven cavity (x zero on the wall faces u(0, j), v(i, 0))."""
        torch = _torch()
        y = torch.empty_like(x) if y is None else y
        self._check(self.lib.sib_cavity_apply_operator(self.ctx, int(l), self._prec(x), _ptr(x), _ptr(y), _stream()))
        return y

    def cavity_smooth(self, l, x, b, sweeps=1):
        """x <- `sweeps` additive Vanka sweeps of the lid-driven cavity, in place."""
        self._check(self.lib.sib_cavity_smooth(self.ctx, int(l), self._prec(x), _ptr(x), _ptr(b), int(sweeps),
                                               _stream()))
        return x

    def apply_ib(self, l, u, f=None):
        torch = _torch()
        f = torch.empty_like(u) if f is None else f
        self._check(self.lib.sib_apply_ib(self.ctx, int(l), self._prec(u), _ptr(u), _ptr(f), _stream()))
        return f

    def smooth(self, l, x, b, sweeps=1):
        self._check(self.lib.sib_smooth(self.ctx, int(l), self._prec(x), _ptr(x), _ptr(b), int(sweeps), _stream()))
        return x

    def residual_restrict(self, l, x, b):
        torch = _torch()
        Nc = self.level_size(l - 1)
        rc = torch.empty(3 * Nc * Nc, dtype=x.dtype, device=x.device)
        self._check(self.lib.sib_residual_restrict(self.ctx, int(l), self._prec(x), _ptr(x), _ptr(b), _ptr(rc),
                                                   _stream()))
        return rc

    def prolong_add(self, l, ec, xf):
        self._check(self.lib.sib_prolong_add(self.ctx, int(l), self._prec(ec), _ptr(ec), _ptr(xf), _stream()))
        return xf

    def coarse_solve(self, b, x=None):
        torch = _torch()
        x = torch.empty_like(b) if x is None else x
        self._check(self.lib.sib_coarse_solve(self.ctx, self._prec(b), _ptr(b), _ptr(x), _stream()))
        return x

    def vcycle(self, b, z=None):
        torch = _torch()
        z = torch.empty_like(b) if z is None else z
        self._check(self.lib.sib_vcycle(self.ctx, self._prec(b), _ptr(b), _ptr(z), _stream()))
        return z

    def interp(self, u):
        torch = _torch()
        U = torch.empty((max(self.M, 1), 2), dtype=torch.float64, device=u.device)[: self.M]
        self._check(self.lib.sib_interp(self.ctx, _ptr(u), _ptr(U) if self.M else None, _stream()))
        return U

    def advance_markers(self, w):
        """X^{n+1} = X^n + dt J^n u^{n+1} for the solution w of the step (Eq. imp-X-new)."""
        torch = _torch()
        Xn = torch.empty((max(self.M, 1), 2), dtype=torch.float64, device=w.device)[: self.M]
        self._check(self.lib.sib_advance_markers(self.ctx, _ptr(w), _ptr(Xn) if self.M else None, _stream()))
        return Xn

    def spread(self, F):
        torch = _torch()
        f = torch.empty(2 * self.N * self.N, dtype=torch.float64, device=F.device)
        self._check(self.lib.sib_spread(self.ctx, _ptr(F) if self.M else None, _ptr(f), _stream()))
        return f

    def time_kernel(self, kernel: str, level: int, fp32: bool, reps: int = 20, cold: bool = False):
        """(mean ms per launch, algorithmic bytes per launch) of one V-cycle kernel, CUDA events.
        cold: no warm-up launch (the caller flushes L2 before the call and times reps = 1)."""
        ms = ctypes.c_double()
        by = ctypes.c_double()
        kid = KERNELS[kernel] | (TIME_COLD if cold else 0)
        self._check(self.lib.sib_time_kernel(self.ctx, kid, int(level), PREC_FP32 if fp32 else PREC_FP64,
                                             int(reps), _stream(), ctypes.byref(ms), ctypes.byref(by)))
        return ms.value, by.value

    @property
    def launch_count(self):
        return int(self.lib.sib_launch_count(self.ctx))

    @property
    def device_bytes(self):
        return int(self.lib.sib_device_bytes(self.ctx))


def time_loop(solver, g, X, edges, kappa, steps):
    """`steps` semi-implicit time steps (Sec. 2.2): set the structure X^n, set up, solve
    L_IB(X^n) w = (g + S K X^n, 0) and move the markers, X^{n+1} = X^n + dt J^n u^{n+1}
    (Eq. imp-X-new).  g is the full momentum right-hand side of every step (steady forcing; with
    rho > 0 a caller that wants the (rho/dt) u^n term puts it into g).  Every step runs in the
    library; this only sequences its calls.  Returns [w^1 ..], [X^0, X^1 ..] (device tensors)."""
    ws, Xs = [], [X]
    for _ in range(steps):
        solver.set_structure(X, edges, kappa)
        solver.setup()
        w = solver.solve(g)
        X = solver.advance_markers(w)
        ws.append(w)
        Xs.append(X)
    return ws, Xs


def solver_for(problem, device="cuda", **opts):
    """Create, configure and set up a Solver for an ``inputs.Problem``."""
    torch = _torch()
    s = Solver(problem.N)
    s.set_fluid(problem.rho, problem.mu, problem.dt)
    st = problem.structure
    X = torch.as_tensor(st.X, dtype=torch.float64, device=device).contiguous()
    E = torch.as_tensor(st.edges, dtype=torch.int32, device=device).contiguous()
    K = torch.as_tensor(st.kappa, dtype=torch.float64, device=device).contiguous()
    s.set_structure(X, E, K)
    if opts:
        s.set_options(**opts)
    s.setup()
    return s

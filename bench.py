#!/usr/bin/env python
"""Benchmark of the differentiated Stokes-IB solve on its largest single-GPU workload.

Headline workload (one step = one differentiated solve): periodic 1024 x 1024 MAC grid, rho = 1,
mu = 1e-2, dt = 1e-3; a thick elastic disk (radius 0.15 at (0.3, 0.5), concentric marker rings at
half-cell spacing) and a thin ellipse (semi-axes 0.15 / 0.10 at (0.7, 0.5)): 298,858 markers and
596,106 zero-rest-length springs, kappa = 1e4; seeded N(0,1) forcing g.  A step is
  1. sib_set_structure (X, springs, kappa) and sib_setup: marker binning, Galerkin IB windows,
     coarsest pseudo-inverse, SC eigenvalue estimates;
  2. the forward solve L_IB w = (g + S K X^n, 0): FP64 FGMRES(100) to a 1e-8 relative residual,
     preconditioned by one FP32 V-cycle with the Schur-complement smoother in the paper's
     FGMRES-wrapped form (Sec. 3.3);
  3. the adjoint solve L_IB^T lam = (2 (u - u*), 0) of the loss ||u - u*||^2 (sib_solve_transpose),
     u* the velocity of a solve with another seeded forcing;
  4. sib_grad: d loss / d kappa (every spring) and d loss / d X (every marker).

Output: one JSON line (rank 0).  `value` is device time per step (ms) over the whole job (every rank
runs its own replica); `e2e` is the same step through the autograd binding with g, kappa and X copied
from pinned host memory and the loss and gradients copied back.  The other workloads of the build
(32^2 to 512^2, the paper's own structures, the lid-driven cavity, the 4096^2 V-cycle roofline) are
reported beside it, each result with its error against the FP64 oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--cpu-breadth]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
if __name__ == "__main__" and "--impl" in sys.argv and "reference" in sys.argv:
    # the reference arm runs the oracle on one thread, like the CPU baseline; numpy's BLAS reads these
    # when it loads, so they are set before the first import of numpy
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

METRIC = "Stokes-IB solve time to 1e-8 rel resid; V-cycle Mdof/s & %HBM; FP32 vs FP64 MG"
WORKLOAD = "disk_and_ellipse_re_N1024_kappa1e4_differentiated"
N_HEAD = 1024
TARGET_SEED = 40            # forcing of the reference solve that gives u*
LARGE_N = 4096
L2_BYTES = 129 * 2 ** 20
KAPPAS = [1e0, 1e2, 1e4, 1e6]
SMOOTHERS = ["vanka", "sc"]
WIDE_BOX = (8, 2)           # the paper's 8 x 8 boxes with overlap 2 (Sec. 5.1.1, 5.2.1)
HUGE_BOX = (16, 4)          # and its 16 x 16 boxes with overlap 4
# FGMRES iterations of the headline's forward and adjoint solves: the oracle's time per iteration is
# scaled by these to the time of one differentiated solve (the CPU baseline is a bounded sample)
HEAD_ITERATIONS = (38, 38)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")
BREADTH_FILE = os.path.join(ROOT, "profiles", "oracle_cpu_baseline_configs0-3.md")
CSRC = os.path.join(ROOT, "paper_1612_02208_gb300", "csrc")
# the source text of each roofline kernel: file, first and last marker (the kernel and its launcher)
KERNEL_SOURCES = {
    "k_ib_window_f32": ("kernels_ib.cu", "struct WinVec;", "template void launch_ib_window<float>"),
    "k_vanka_f32": ("kernels_grid.cu", "k_vanka_pair(GridK<T> g", "// Tensor map of a level vector"),
}


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-large", action="store_true", help="skip the 4096^2 V-cycle roofline leg")
    p.add_argument("--no-paper", action="store_true", help="skip the paper-workload and cavity tables")
    p.add_argument("--quick", action="store_true", help="headline only (no other legs)")
    p.add_argument("--large-n", type=int, default=LARGE_N, help="grid of the large-grid V-cycle roofline")
    p.add_argument("--profile-setup", action="store_true",
                   help="the headline's set-up twice inside an NVTX range (for an ncu launch list)")
    p.add_argument("--profile-vcycle", choices=["headline", "large", "large64", "large2k", "ras16", "ras8o2"], default=None,
                   help="two FP32 V-cycles in an NVTX range 'vcycle', with a one-vector FGMRES basis (the small-memory "
                        "case for ncu captures): 'headline' = the headline workload and smoother, 'large' = the "
                        "4096^2 thin ellipse with Vanka, 'large64' = the same body on 2048^2 with the FP64 V-cycle, "
                        "'ras8o2' = the 2048^2 grid without a structure, RAS with "
                        "8 x 8 boxes of overlap 2 corrected on the tensor cores")
    p.add_argument("--profile-solve", action="store_true",
                   help="one FGMRES solve of the 128^2 disk (Vanka, kappa = 1e2) without CUDA graphs, in an NVTX range "
                        "'solve', so that ncu lists the Krylov kernels that the device graph otherwise hides")
    p.add_argument("--cpu-breadth", action="store_true",
                   help="time the oracle on configurations 0-3 (direct and FGMRES, 1 thread and all threads) "
                        "and write the table (--breadth-out, default under profiles/)")
    p.add_argument("--breadth-out", default=BREADTH_FILE, help="where --cpu-breadth writes its table")
    return p.parse_args(argv)


# ------------------------------------------------------------------------------------ ranks
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def dist_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def dist_max(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_ms_per_unit(max_time_ms: float, units_per_rank: int, world: int) -> float:
    """Whole-job time per unit: the slowest rank's time over the units all ranks completed."""
    return max_time_ms / float(units_per_rank * world)


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.proc = None
        self.index = index
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = [ln.strip().split(",") for ln in open(self.path) if ln.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 3 + k and r[3 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------ peaks / traffic
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash(kernel: str):
    """Hash of the kernel's source text (its definition and launcher): a recorded capture is valid only
    while that text is unchanged."""
    fname, first, last = KERNEL_SOURCES[kernel]
    text = open(os.path.join(CSRC, fname)).read()
    i = text.index(first)
    return hashlib.sha256(text[i:text.index(last, i)].encode()).hexdigest()[:12]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    h = source_hash(kernel)
    for line in open(TRAFFIC_FILE):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == workload and f[3] == h:
            return float(f[2])
    return None


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ------------------------------------------------------------------------------------ native arm
def stats_record(S, **extra):
    d = S.stats.as_dict()
    rec = dict(iterations=d["iterations"], converged=d["converged"], rel_residual=d["rel_residual"],
               setup_ms=round(d["setup_ms"], 4), solve_ms=round(d["solve_ms"], 4))
    rec.update(extra)
    return rec


class Headline:
    """The differentiated solve of the headline workload, on device tensors."""

    def __init__(self, sib, torch, dev):
        from paper_1612_02208_gb300 import inputs
        self.sib, self.torch, self.dev = sib, torch, dev
        self.prob = inputs.disk_and_ellipse_re(N_HEAD)
        st = self.prob.structure
        self.n = N_HEAD * N_HEAD
        self.S = sib.Solver(N_HEAD)
        self.S.set_fluid(self.prob.rho, self.prob.mu, self.prob.dt)
        self.X = torch.as_tensor(st.X, device=dev)
        self.E = torch.as_tensor(st.edges, device=dev)
        self.kap = torch.as_tensor(st.kappa, device=dev)
        self.g = torch.as_tensor(self.prob.g, device=dev)
        self.w = torch.empty_like(self.g)
        self.lam = torch.empty_like(self.g)
        self.adj = torch.zeros_like(self.g)
        self.set_options()
        # u*: the velocity of a solve with another seeded forcing
        self.S.set_structure(self.X, self.E, self.kap)
        self.S.setup()
        gt = torch.as_tensor(inputs.forcing(N_HEAD, TARGET_SEED), device=dev)
        self.ustar = self.S.solve(gt)[: 2 * self.n].clone()
        self.events = None

    def set_options(self, **kw):
        o = dict(smoother=self.sib.SMOOTHER_SC, smooth_krylov=1, sc_relax=self.sib.RELAX_JACOBI, vcycle_fp32=1,
                 omega=-1.0, rtol=1e-8, max_it=100, restart=100)
        o.update(kw)
        self.S.set_options(**o)

    def step(self, stream, record=False, forward_only=False):
        torch, S = self.torch, self.S
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)] if record else None
        if ev:
            ev[0].record(stream)
        S.set_structure(self.X, self.E, self.kap)
        S.setup()
        if ev:
            ev[1].record(stream)
        S.solve(self.g, self.w, allow_unconverged=True)
        fwd = stats_record(S) if record else None
        if ev:
            ev[2].record(stream)
        if forward_only:
            return fwd, None, None
        self.adj[: 2 * self.n] = 2.0 * (self.w[: 2 * self.n] - self.ustar)
        S.solve_transpose(self.adj, self.lam, allow_unconverged=True)
        adj = stats_record(S) if record else None
        if ev:
            ev[3].record(stream)
        dk, dX = S.grad(self.w, self.lam)
        if ev:
            ev[4].record(stream)
            ev[4].synchronize()
            self.events = dict(setup_ms=ev[0].elapsed_time(ev[1]), forward_ms=ev[1].elapsed_time(ev[2]),
                               adjoint_ms=ev[2].elapsed_time(ev[3]), grad_ms=ev[3].elapsed_time(ev[4]))
        return fwd, adj, (dk, dX)


def headline_e2e(H, sib, torch, steps):
    """The step through the autograd binding: g, kappa and X copied from pinned host memory, the loss
    and the gradients copied back, every step; wall-clock time around the steps."""
    from paper_1612_02208_gb300 import autograd
    prob, dev = H.prob, H.dev
    st = prob.structure
    g_h = torch.as_tensor(prob.g).pin_memory()
    k_h = torch.as_tensor(st.kappa).pin_memory()
    X_h = torch.as_tensor(st.X).pin_memory()
    dk_h = torch.empty_like(k_h).pin_memory()
    dX_h = torch.empty_like(X_h).pin_memory()
    loss_h = torch.empty(1, dtype=torch.float64).pin_memory()
    n = H.n

    def one():
        g = g_h.to(dev, non_blocking=True)
        kap = k_h.to(dev, non_blocking=True).requires_grad_(True)
        X = X_h.to(dev, non_blocking=True).requires_grad_(True)
        w = autograd.stokes_ib_solve(H.S, g, kap, X, H.E)
        loss = ((w[: 2 * n] - H.ustar) ** 2).sum()
        loss.backward()
        dk_h.copy_(kap.grad, non_blocking=True)
        dX_h.copy_(X.grad, non_blocking=True)
        loss_h.copy_(loss.detach().reshape(1), non_blocking=True)
        torch.cuda.current_stream().synchronize()

    one()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t) * 1e3 / steps
    h2d = 8 * (g_h.numel() + k_h.numel() + X_h.numel())
    d2h = 8 * (dk_h.numel() + dX_h.numel() + 1)
    return ms, h2d, d2h


def headline_variants(H, stream):
    """Beside the headline (same workload, one run each): SC with damped sweeps (the library default)
    and the headline's solve with an all-FP64 V-cycle (FP32 against FP64 multigrid)."""
    out = {}
    H.set_options(smooth_krylov=0)
    f, _, _ = H.step(stream, record=True, forward_only=True)
    out["sc_damped_fp32_forward"] = f
    H.set_options(vcycle_fp32=0)
    f, a, _ = H.step(stream, record=True)
    out["sc_wrapped_fp64_vcycle"] = {"forward": f, "adjoint": a, "phases_ms": dict(H.events)}
    H.set_options()
    return out


def solve_case(sib, torch, prob, dev, keep=True, **opts):
    """One forward solve of an inputs.Problem; returns (record, w on the host)."""
    S = sib.solver_for(prob, device=dev, **opts)
    g = torch.as_tensor(prob.g, device=dev)
    w = S.solve(g, allow_unconverged=True)
    torch.cuda.synchronize()
    rec = stats_record(S)
    S.close()
    return rec, (w.cpu().numpy() if keep else None)


def config_legs(sib, torch, dev, stream, keep):
    """Configurations 0-3 beside the headline.  keep collects (problem, w) pairs for the oracle checks."""
    from paper_1612_02208_gb300 import inputs
    out = {}
    # configuration 0: 32^2 thin ellipse, Stokes, Vanka
    p0 = inputs.thin_ellipse_stokes(32)
    rec, w = solve_case(sib, torch, p0, dev)
    keep.append(("config0", p0, w, "direct"))
    out["config0_ellipse32_vanka"] = rec
    # configuration 1: the 128^2 disk, kappa sweep x {Vanka, SC}, FP32 and FP64 V-cycles, plus the
    # paper's smoothing forms
    out["config1_disk128"] = disk128_legs(sib, torch, dev, stream, keep)
    # configuration 2: 512^2 thin ellipse, rho = 1; FP32 V-cycle inside FP64 FGMRES against all-FP64
    c2 = []
    for kap in (1e2, 1e4):
        prob = inputs.thin_ellipse_re(512, kappa=kap)
        for fp32 in (1, 0):
            rec, w = solve_case(sib, torch, prob, dev, vcycle_fp32=fp32)
            keep.append((f"config2_kappa{kap:g}_fp{32 if fp32 else 64}", prob, w, "residual"))
            c2.append(dict(kappa=kap, vcycle="fp32" if fp32 else "fp64", **rec))
    out["config2_ellipse512_re"] = c2
    # configuration 3: 256^2 thin ellipse with LogUniform(1e2, 1e4) stiffness, differentiated solve
    out["config3_ellipse256_loguniform"] = config3_leg(sib, torch, dev, keep)
    return out


def disk128_legs(sib, torch, dev, stream, keep):
    from paper_1612_02208_gb300 import inputs
    prob = inputs.disk_stokes(128, kappa=1.0, seed=1)
    st = prob.structure
    S = sib.Solver(prob.N)
    S.set_fluid(prob.rho, prob.mu, prob.dt)
    S.set_structure(torch.as_tensor(st.X, device=dev), torch.as_tensor(st.edges, device=dev),
                    torch.as_tensor(st.kappa, device=dev))
    kap_dev = {k: torch.full((st.E,), k, dtype=torch.float64, device=dev) for k in KAPPAS}
    g = torch.as_tensor(prob.g, device=dev)
    w = torch.empty_like(g)
    forms = {
        "damped": dict(smooth_krylov=0),
        "fp64_vcycle": dict(vcycle_fp32=0),
        "wrapped": dict(smooth_krylov=1),
    }
    out = {}
    for form, extra in forms.items():
        recs = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sm in SMOOTHERS:
            o = dict(smoother=sib.SMOOTHER_SC if sm == "sc" else sib.SMOOTHER_VANKA, omega=-1.0, vcycle_fp32=1,
                     smooth_krylov=0, sc_relax=sib.RELAX_JACOBI)
            o.update(extra)
            S.set_options(**o)
            for kap in KAPPAS:
                S.set_stiffness(kap_dev[kap])
                S.setup()
                S.solve(g, w, allow_unconverged=True)
                recs.append(stats_record(S, smoother=sm, kappa=kap))
                if form == "damped":
                    keep.append((f"config1_{sm}_kappa{kap:g}", (prob, kap), w.cpu().numpy(), "direct"))
        e1.record(stream)
        e1.synchronize()
        out[form] = {"ms_per_solve": round(e0.elapsed_time(e1) / len(recs), 4), "cases": recs}
    # SC with symmetric red-black Gauss-Seidel in its Chebyshev iterations (Sec. 3.3, SC smoothing)
    recs = []
    S.set_options(smoother=sib.SMOOTHER_SC, vcycle_fp32=1, omega=-1.0, smooth_krylov=0, sc_relax=sib.RELAX_SGS)
    for kap in KAPPAS:
        S.set_stiffness(kap_dev[kap])
        S.setup()
        S.solve(g, w, allow_unconverged=True)
        recs.append(stats_record(S, kappa=kap))
    out["sc_gauss_seidel"] = recs
    # box RAS (Sec. 3.3, Alg. 2 with boxes): 4 x 4 and 2 x 2 boxes with overlap 1, the paper's 8 x 8 with 2
    ras = []
    for b, o in ((4, 1), (2, 1), WIDE_BOX):
        S.set_options(smoother=sib.SMOOTHER_RAS, sc_relax=sib.RELAX_JACOBI, box=b, box_overlap=o, omega=-1.0)
        for kap in KAPPAS:
            S.set_stiffness(kap_dev[kap])
            S.setup()
            S.solve(g, w, allow_unconverged=True)
            ras.append(stats_record(S, box=b, overlap=o, kappa=kap))
    out["box_ras"] = ras
    S.close()
    return out


def config3_leg(sib, torch, dev, keep):
    """Differentiated solve of the 256^2 LogUniform-stiffness ellipse (loss ||u - u*||^2, u* from a solve
    with an independently seeded stiffness), FP64 and FP32-preconditioned."""
    from paper_1612_02208_gb300 import inputs
    prob = inputs.thin_ellipse_loguniform(256)
    other = inputs.thin_ellipse_loguniform(256, seed_kappa=30)
    n = prob.N ** 2
    out = []
    for fp32 in (0, 1):
        S = sib.solver_for(other, device=dev, vcycle_fp32=fp32)
        ustar = S.solve(torch.as_tensor(other.g, device=dev))[: 2 * n].clone()
        S.set_stiffness(torch.as_tensor(prob.structure.kappa, device=dev))
        S.setup()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        w = S.solve(torch.as_tensor(prob.g, device=dev), allow_unconverged=True)
        fwd = stats_record(S)
        adj = torch.zeros_like(w)
        adj[: 2 * n] = 2.0 * (w[: 2 * n] - ustar)
        lam = S.solve_transpose(adj, allow_unconverged=True)
        bwd = stats_record(S)
        dk, dX = S.grad(w, lam)
        e1.record()
        e1.synchronize()
        key = f"config3_fp{32 if fp32 else 64}"
        keep.append((key, prob, w.cpu().numpy(), "residual"))
        keep.append((key + "_grad", prob, (w.cpu().numpy(), lam.cpu().numpy(), dk.cpu().numpy(), dX.cpu().numpy()),
                     "gradient"))
        out.append(dict(vcycle="fp32" if fp32 else "fp64", ms=round(e0.elapsed_time(e1), 4), forward=fwd,
                        adjoint=bwd))
        S.close()
    return out


def paper_workloads(sib, torch, dev):
    """The paper's thick annulus and thin circle (Sec. 5.1, 5.2) in the periodic box: one linear solve
    each (dt = 0.32 h, g = 0, tolerance 1e-12, at most 100 iterations, FP32 V-cycle), over gamma,
    Stokes and mu = 0.01, and the smoothers; plus the annulus under grid refinement."""
    from paper_1612_02208_gb300 import inputs
    smoothers = {"vanka": dict(smoother=sib.SMOOTHER_VANKA), "sc": dict(smoother=sib.SMOOTHER_SC),
                 "ras4o1": dict(smoother=sib.SMOOTHER_RAS, box=4, box_overlap=1),
                 "ras2o2": dict(smoother=sib.SMOOTHER_RAS, box=2, box_overlap=2),
                 "ras8o2": dict(smoother=sib.SMOOTHER_RAS, box=WIDE_BOX[0], box_overlap=WIDE_BOX[1]),
                 "ras16o4": dict(smoother=sib.SMOOTHER_RAS, box=HUGE_BOX[0], box_overlap=HUGE_BOX[1])}
    runs = [(kind, 128, gamma, mu, sm) for kind in ("annulus", "circle") for mu in (None, 0.01)
            for gamma in (5.0, 50.0, 500.0) for sm in smoothers]
    runs += [("annulus", N, gamma, None, sm) for N in (64, 256) for gamma in (5.0, 500.0) for sm in ("vanka", "ras4o1")]
    runs += [("circle", N, 500.0, None, sm) for N in (64, 256) for sm in ("ras8o2", "ras16o4")]
    cases = []
    for kind, N, gamma, mu, sm in runs:
        prob = inputs.paper_problem(kind, N, gamma, mu)
        st = prob.structure
        S = sib.Solver(N)
        S.set_fluid(prob.rho, prob.mu, prob.dt)
        S.set_structure(torch.as_tensor(st.X, device=dev), torch.as_tensor(st.edges, device=dev),
                        torch.as_tensor(st.kappa, device=dev))
        S.set_options(rtol=1e-12, max_it=100, **smoothers[sm])
        S.setup()
        g = torch.zeros(3 * N * N, dtype=torch.float64, device=dev)
        w = torch.empty_like(g)
        S.solve(g, w, allow_unconverged=True)
        d = S.stats.as_dict()
        cases.append(dict(kind=kind, N=N, gamma=gamma, flow="stokes" if mu is None else f"mu={mu}", smoother=sm,
                          iterations=d["iterations"], converged=d["converged"], setup_ms=round(d["setup_ms"], 3),
                          solve_ms=round(d["solve_ms"], 3)))
        S.close()
    return {"tol": 1e-12, "max_it": 100, "dt": "0.32 h", "g": "0 (elastic force of the initial configuration)",
            "boundary": "periodic", "cases": cases}


def cavity_workloads(sib, torch, dev):
    """The paper's lid-driven cavity (Sec. 5: no-slip walls, regularised lid) with its thick annulus and
    thin circle, Stokes flow, one linear solve each (dt = 0.32 h, g = 0: the lid and the elastic force
    of the initial configuration drive the flow; tolerance 1e-12, at most 100 iterations, FP32 V-cycle,
    Vanka), over gamma."""
    from paper_1612_02208_gb300 import inputs
    cases = []
    for kind in ("annulus", "circle"):
        for gamma in (5.0, 50.0, 500.0):
            prob = inputs.paper_problem(kind, 128, gamma)
            st = prob.structure
            S = sib.Solver(prob.N)
            S.set_fluid(prob.rho, prob.mu, prob.dt)
            S.set_structure(torch.as_tensor(st.X, device=dev), torch.as_tensor(st.edges, device=dev),
                            torch.as_tensor(st.kappa, device=dev))
            S.set_options(domain=sib.DOMAIN_CAVITY, rtol=1e-12, max_it=100)
            S.setup()
            g = torch.zeros(3 * prob.N * prob.N, dtype=torch.float64, device=dev)
            w = torch.empty_like(g)
            S.solve(g, w, allow_unconverged=True)
            d = S.stats.as_dict()
            cases.append(dict(kind=kind, N=prob.N, gamma=gamma, flow="stokes", smoother="vanka",
                              iterations=d["iterations"], converged=d["converged"],
                              setup_ms=round(d["setup_ms"], 3), solve_ms=round(d["solve_ms"], 3)))
            S.close()
    return {"tol": 1e-12, "max_it": 100, "dt": "0.32 h", "boundary": "lid-driven cavity", "cases": cases}


def large_vcycle(sib, torch, reps=20, N=None):
    """V-cycle throughput and the grid kernels' rooflines on a grid whose working set exceeds L2
    (4096^2: one FP32 sweep moves 600 MB), rho = 1, mu = 1e-2, dt = 1e-3, thin ellipse, kappa = 1e4,
    FP32 V-cycle; Vanka, then box RAS (4 x 4 boxes, overlap 1; 8 x 8, overlap 2)."""
    from paper_1612_02208_gb300 import inputs
    LARGE = N or LARGE_N
    prob = inputs.thin_ellipse_re(LARGE, kappa=1e4, seed=2)
    S = sib.Solver(LARGE)
    S.set_fluid(prob.rho, prob.mu, prob.dt)
    st = prob.structure
    dev = torch.device("cuda")
    S.set_structure(torch.as_tensor(st.X, device=dev), torch.as_tensor(st.edges, device=dev),
                    torch.as_tensor(st.kappa, device=dev))
    S.set_options(restart=1, max_it=1)
    S.setup()
    n3 = 3 * LARGE * LARGE
    b = torch.randn(n3, device=dev, dtype=torch.float32)
    z = torch.empty_like(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_cycles():
        for _ in range(3):
            S.vcycle(b, z)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            S.vcycle(b, z)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_v = time_cycles()
    lmax = S.num_levels - 1
    out = {"workload": f"thin_ellipse_re_N{LARGE}_kappa1e4", "N": LARGE, "vcycle_ms": round(t_v, 4),
           "vcycle_mdofs": round(n3 / (t_v * 1e-3) / 1e6, 1), "kernels": {}}
    for name in ("vanka", "residual", "restrict", "residual_restrict", "prolong", "interp", "spread"):
        ms, by = S.time_kernel(name, lmax, True, reps=20)
        out["kernels"][name] = {"ms": round(ms, 5), "bytes": by, "gbs": round(by / (ms * 1e-3) / 1e9, 1)}
    for (bx, ov), key in (((4, 1), "ras"), (WIDE_BOX, "ras8o2")):
        S.set_options(smoother=sib.SMOOTHER_RAS, box=bx, box_overlap=ov, omega=-1.0, ras_tc=1)
        S.setup()
        # the correction is a dense product: 2 ne flops per owned dof, ne = 3 e^2 + 2 e, e = b + 2 o
        e = bx + 2 * ov
        flops = 2.0 * (3 * e * e + 2 * e) * 3.0 * LARGE * LARGE
        for tc, suffix in ((1, ""), (0, "_cuda_cores")):
            S.set_options(ras_tc=tc)
            out["vcycle_ms_" + key + suffix] = round(time_cycles(), 4)
            ms, by = S.time_kernel("ras", lmax, True, reps=20)
            out["kernels"][key + suffix] = {"ms": round(ms, 5), "bytes": by, "gbs": round(by / (ms * 1e-3) / 1e9, 1),
                                            "tflops": round(flops / (ms * 1e-3) / 1e12, 2)}
        S.set_options(ras_tc=1)
    S.close()
    return out


def time_loop_leg(sib, torch, dev, steps=5):
    """The semi-implicit time loop on the 128^2 disk (Vanka, kappa = 1e2): every step sets the
    structure at X^n, sets up, solves to 1e-8 and moves the markers, X^{n+1} = X^n + dt J^n u^{n+1}.
    Timed by CUDA events around the loop (the set-up's host synchronisations included)."""
    from paper_1612_02208_gb300 import inputs
    prob = inputs.disk_stokes(128, kappa=1e2, seed=1)
    st = prob.structure
    S = sib.Solver(prob.N)
    S.set_fluid(prob.rho, prob.mu, prob.dt)
    X = torch.as_tensor(st.X, device=dev)
    E = torch.as_tensor(st.edges, device=dev)
    kap = torch.full((st.E,), 1e2, dtype=torch.float64, device=dev)
    g = torch.as_tensor(prob.g, device=dev)
    sib.time_loop(S, g, X, E, kap, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ws, Xs = sib.time_loop(S, g, X, E, kap, steps)
    e1.record()
    e1.synchronize()
    out = {"workload": "disk_stokes_N128_kappa1e2_vanka", "steps": steps,
           "ms_per_time_step": round(e0.elapsed_time(e1) / steps, 4),
           "max_marker_displacement": float((Xs[-1] - Xs[0]).abs().max())}
    S.close()
    return out


def dominant_kernel_roofline(H, peak, peak_kind, flush, reps=20):
    """The step's dominant kernel: the IB window pass of the finest level (FP32; four in every SC sweep
    and one before every operator application of the V-cycle), timed by CUDA events on the headline's
    own context and stream, each launch after an L2 flush (its windows, 73 MB, would otherwise stay in
    L2 between back-to-back launches).  Algorithmic bytes per launch: 15 words per marker plus 2 words
    per IB-touched face (the IB operator applied through the markers)."""
    torch = H.torch
    lmax = H.S.num_levels - 1
    cold = []
    for r in range(reps):
        flush.fill_(float(r))
        ms, by = H.S.time_kernel("ib_window", lmax, True, reps=1, cold=True)
        cold.append(ms)
    ms = float(np.mean(cold))
    warm_ms, _ = H.S.time_kernel("ib_window", lmax, True, reps=reps)
    torch.cuda.synchronize()
    achieved = by / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": "k_ib_window<float> (finest level, 1024^2)", "achieved": round(achieved, 1),
            "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": recorded_traffic("k_ib_window_f32", WORKLOAD), "bytes_per_launch": by,
            "launch_ms": round(ms, 5), "launch_ms_l2_warm": round(warm_ms, 5), "peak_source": peak_kind,
            "timing": "mean of 20 launches, each after an L2 flush"}


def run_native(args):
    import torch
    from paper_1612_02208_gb300 import sib

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    rank, world = dist_init("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    H = Headline(sib, torch, dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(max(args.warmup, 0)):
        H.step(stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    dist_barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("timed_steps")
    launches0 = H.S.launch_count
    step_ms, phases, first = [], [], None
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                     # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fwd, adj, _ = H.step(stream, record=True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        phases.append(H.events)
        if first is None:
            first = {"forward": fwd, "adjoint": adj}
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dist_barrier()
    wall = time.perf_counter() - t_wall
    launches = H.S.launch_count - launches0
    clk = clocks.stop()
    total_ms = float(sum(step_ms))
    max_total = dist_max(total_ms, dev)
    value = job_ms_per_unit(max_total, args.steps, world)
    phase_ms = {k: round(float(np.median([p[k] for p in phases])), 4) for k in phases[0]}

    # the dominant kernel, timed live on the headline's context and stream
    peak, peak_kind = measured_peaks()
    roofline = dominant_kernel_roofline(H, peak, peak_kind, flush)

    # the headline's results for the oracle checks (gradient and residuals)
    H.step(stream)
    torch.cuda.synchronize()
    dk, dX = H.S.grad(H.w, H.lam)
    head_keep = (H.prob, H.w.cpu().numpy(), H.lam.cpu().numpy(), H.adj.cpu().numpy(), dk.cpu().numpy(),
                 dX.cpu().numpy())

    # end to end through the autograd binding, pinned host memory
    e2e_steps = max(1, min(args.steps, 3))
    e2e_ms, h2d, d2h = headline_e2e(H, sib, torch, e2e_steps)
    e2e_value = job_ms_per_unit(dist_max(e2e_ms * e2e_steps, dev), e2e_steps, world)
    e2e = {"value": round(e2e_value, 4), "unit": "ms/step", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h)}

    variants = headline_variants(H, stream) if not args.quick else None
    H.S.close()

    keep = []
    legs = {}
    if not args.quick:
        legs.update(config_legs(sib, torch, dev, stream, keep))
        if not args.no_paper:
            legs["paper_workloads"] = paper_workloads(sib, torch, dev)
            legs["cavity_workloads"] = cavity_workloads(sib, torch, dev)
        legs["time_loop"] = time_loop_leg(sib, torch, dev)
        if not args.no_large:
            large = large_vcycle(sib, torch, N=args.large_n)
            large["roofline_vanka"] = {"achieved": large["kernels"]["vanka"]["gbs"], "peak": peak,
                                       "frac": round(large["kernels"]["vanka"]["gbs"] / peak, 4),
                                       "traffic": recorded_traffic("k_vanka_f32", large["workload"])}
            legs["vcycle_large"] = large

    cpu, checks = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, checks = oracle_leg(head_keep, keep)

    if rank == 0:
        st = H.prob.structure
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "ms/step", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(max_total / args.steps, 4), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_HEAD, "markers": st.M, "springs": st.E, "kappa": 1e4,
                       "rho": H.prob.rho, "mu": H.prob.mu, "dt": H.prob.dt,
                       "step": "set structure + set-up, forward solve, adjoint solve, gradients (kappa, X)",
                       "smoother": "Schur complement, FGMRES-wrapped sweeps (nu1 = nu2 = 2)",
                       "vcycle": "fp32, coarsest fp64", "krylov": "fp64 FGMRES(100), CGS2", "rtol": 1e-8,
                       "max_it": 100, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (inputs exceed L2: FGMRES basis 2.5 GB)",
                       "timing": "CUDA events per step on the launching stream"},
            "headline": {"first_timed_step": first, "phase_ms_median": phase_ms,
                         "oracle_checks": checks.get("headline") if checks else None},
            "variants": variants, "legs": legs,
            "oracle_checks": checks.get("legs") if checks else None,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk, "wall_s": round(wall, 3),
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------ the oracle
# Everything below runs the CPU oracle (oracle/): the CPU baseline, the reference arm and the oracle's
# checks of the GPU results.  It is test infrastructure, never on the product path.
def _rel(a, b):
    s = float(np.abs(b).max())
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


def _oracle_matvec(prob, w):
    """L_IB w through the oracle's sparse pieces (A, G, D, J, K, S = J^T / h^2)."""
    from oracle import ib, mac
    N, s = prob.N, prob.structure
    n = N * N
    u, p = w[:2 * n], w[2 * n:]
    K = ib.stiffness(s.X.shape[0], s.edges, s.kappa)
    f = np.concatenate([ib.spread_matrix(N, s.X, c) @ (K @ (ib.interp_matrix(N, s.X, c) @ u[c * n:(c + 1) * n]))
                        for c in (0, 1)])
    mom = mac.momentum(N, prob.rho, prob.mu, prob.dt) @ u - prob.dt * f + mac.gradient(N) @ p
    return np.concatenate([mom, -(mac.divergence(N) @ u)])


def _oracle_residual(prob, w, b=None):
    from oracle import system
    b = system.rhs(prob) if b is None else b
    return float(np.linalg.norm(b - _oracle_matvec(prob, w)) / np.linalg.norm(b))


def _direct_solution(item):
    """The oracle's gauge-fixed direct solve of a (problem or (problem, kappa)) item (pool worker)."""
    from oracle import system
    prob = item
    if isinstance(item, tuple):
        prob, kap = item
        prob.structure.kappa[:] = kap
    L = system.operator_of(prob)
    w, _ = system.solve_direct(L, system.rhs(prob), prob.N, prob.rho)
    return system.project(w, prob.N, prob.rho)


def oracle_leg(head_keep, keep):
    """The CPU-baseline leg: the oracle timed on a bounded sample of the headline workload, and the
    oracle's checks of every GPU result kept by the legs (direct solves where affordable, otherwise the
    oracle's residual of the GPU solution; gradients by the oracle's adjoint formula)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from oracle import adjoint, system
    checks = {"legs": {}}
    direct = [(k, p, w) for (k, p, w, kind) in keep if kind == "direct"]
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=max(1, min(8, len(direct))), mp_context=ctx) as ex:
        futs = {k: ex.submit(_direct_solution, p) for k, p, _ in direct}
        # headline: oracle residuals of the forward and adjoint solutions, oracle gradient formula
        prob, w, lam, adj_rhs, dk, dX = head_keep
        t = time.perf_counter()
        rk, rX, _ = adjoint.gradients(prob, w, lam)
        head = {"forward_residual_oracle": _oracle_residual(prob, w),
                "adjoint_residual_oracle": _oracle_residual(prob, lam, adj_rhs),
                "dkappa_rel_err_vs_oracle_formula": _rel(dk, rk), "dX_rel_err_vs_oracle_formula": _rel(dX, rX),
                "note": "oracle's matrix-free residual ||b - L w|| / ||b|| of the GPU's w and lam, and its adjoint "
                        "gradient formula evaluated on them (a direct solve at 1024^2 is unaffordable on the CPU)",
                "seconds": round(time.perf_counter() - t, 2)}
        checks["headline"] = head
        for key, p, w_, kind in keep:
            if kind == "residual":
                checks["legs"][key] = {"oracle_residual": _oracle_residual(p, w_)}
            elif kind == "gradient":
                wg, lg, dkg, dXg = w_
                rk, rX, _ = adjoint.gradients(p, wg, lg)
                checks["legs"][key] = {"dkappa_rel_err_vs_oracle_formula": _rel(dkg, rk),
                                       "dX_rel_err_vs_oracle_formula": _rel(dXg, rX)}
        for key, p, w_ in direct:
            ref = futs[key].result()
            pp = p[0] if isinstance(p, tuple) else p
            checks["legs"][key] = {"err_vs_oracle_direct": _rel(system.project(w_, pp.N, pp.rho), ref)}
    cpu = cpu_baseline_sample()
    return cpu, checks


def _single_thread_env():
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    return env


def oracle_headline_sample(iters=1):
    """The oracle on the headline workload: set-up (operator, right-hand side, SC hierarchy), `iters`
    FGMRES iterations' worth of V-cycles and operator applications, and the gradient formula.  Returns
    the timings and the time of one differentiated solve scaled from them by HEAD_ITERATIONS."""
    from oracle import adjoint, multigrid, system
    from paper_1612_02208_gb300 import inputs
    prob = inputs.disk_and_ellipse_re(N_HEAD)
    t0 = time.perf_counter()
    L = system.operator_of(prob)
    b = system.rhs(prob)
    Hh = multigrid.Hierarchy(prob, smoother="sc", krylov=True)
    t_setup = time.perf_counter() - t0
    per = []
    z = b
    for _ in range(iters):
        t = time.perf_counter()
        z = Hh.vcycle(b)
        y = L @ z
        per.append(time.perf_counter() - t)
    t = time.perf_counter()
    adjoint.gradients(prob, z, y)
    t_grad = time.perf_counter() - t
    t_iter = float(np.median(per))
    ms = (t_setup + t_grad + (HEAD_ITERATIONS[0] + HEAD_ITERATIONS[1]) * t_iter) * 1e3
    return {"ms_per_step": ms, "setup_s": t_setup, "iteration_s": t_iter, "grad_s": t_grad, "iters": iters}


def _sample_worker(iters):
    return oracle_headline_sample(iters)


def cpu_baseline_sample():
    """The oracle on one thread (a fresh process with one BLAS/OpenMP thread), on a bounded sample of
    the headline workload, scaled to ms per differentiated solve."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    old = dict(os.environ)
    os.environ.update({k: v for k, v in _single_thread_env().items() if k.endswith("_NUM_THREADS")})
    try:
        with ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn")) as ex:
            r = ex.submit(_sample_worker, 2).result()
    finally:
        os.environ.clear()
        os.environ.update(old)
    cpu = {"value": round(r["ms_per_step"], 1), "unit": "ms/step", "cores": 1, "kind": "oracle",
           "sample": (f"headline workload, numpy/scipy FP64: set-up (operator, SC hierarchy) {r['setup_s']:.1f} s, "
                      f"{r['iters']} FGMRES iterations' V-cycle + operator application ({r['iteration_s']:.2f} s "
                      f"each, median), gradient formula {r['grad_s']:.1f} s; scaled to "
                      f"{HEAD_ITERATIONS[0]} + {HEAD_ITERATIONS[1]} iterations of one differentiated solve"),
           "nproc": os.cpu_count(), "cpu_model": cpu_model()}
    br = read_breadth()
    if br is not None:
        cpu["breadth"] = br
    return cpu


def read_breadth():
    """The committed table of oracle timings on configurations 0-3 (written by --cpu-breadth)."""
    if not os.path.exists(BREADTH_FILE):
        return None
    text = open(BREADTH_FILE).read()
    for line in text.splitlines():
        if line.startswith("{") and line.rstrip().endswith("}"):
            try:
                d = json.loads(line)
                d["source"] = os.path.relpath(BREADTH_FILE, ROOT)
                return d
            except ValueError:
                return None
    return None


def _breadth_case(name):
    """One configuration of the breadth table, in this process (its thread count set by the caller)."""
    from oracle import krylov, multigrid, system
    from paper_1612_02208_gb300 import inputs
    makers = {
        "config0_ellipse32_vanka": (lambda: inputs.thin_ellipse_stokes(32), "vanka", True),
        "config1_disk128_kappa1e2_vanka": (lambda: inputs.disk_stokes(128, kappa=1e2, seed=1), "vanka", True),
        "config1_disk128_kappa1e2_sc": (lambda: inputs.disk_stokes(128, kappa=1e2, seed=1), "sc", False),
        "config2_ellipse512_re_kappa1e2_vanka": (lambda: inputs.thin_ellipse_re(512, kappa=1e2), "vanka", False),
        "config3_ellipse256_loguniform_vanka": (lambda: inputs.thin_ellipse_loguniform(256), "vanka", True),
    }
    mk, sm, do_direct = makers[name]
    prob = mk()
    out = {"case": name}
    t = time.perf_counter()
    L = system.operator_of(prob)
    b = system.rhs(prob)
    Hh = multigrid.Hierarchy(prob, smoother=sm)
    out["setup_s"] = round(time.perf_counter() - t, 3)
    t = time.perf_counter()
    _, its, _, conv = krylov.fgmres(lambda z: L @ z, Hh.vcycle, b, rtol=1e-8, max_it=100,
                                    project=lambda z: system.project(z, prob.N, prob.rho))
    out.update(fgmres_s=round(time.perf_counter() - t, 3), iterations=its, converged=bool(conv))
    if do_direct:
        t = time.perf_counter()
        system.solve_direct(L, b, prob.N, prob.rho)
        out["direct_s"] = round(time.perf_counter() - t, 3)
    else:
        out["direct_s"] = None
    return out


def run_cpu_breadth(out=BREADTH_FILE):
    """Times the oracle on configurations 0-3 with one thread and with every thread (each case in a
    fresh process), and writes the table (by default under profiles/)."""
    cases = ["config0_ellipse32_vanka", "config1_disk128_kappa1e2_vanka", "config1_disk128_kappa1e2_sc",
             "config3_ellipse256_loguniform_vanka", "config2_ellipse512_re_kappa1e2_vanka"]
    rows = []
    for threads in ("1", "all"):
        env = _single_thread_env() if threads == "1" else dict(os.environ)
        for c in cases:
            code = (f"import sys, json; sys.path.insert(0, {ROOT!r}); import bench; "
                    f"print(json.dumps(bench._breadth_case({c!r})))")
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
            rec = json.loads(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else {"case": c,
                                                                                          "error": r.stderr[-300:]}
            rec["threads"] = threads
            rows.append(rec)
            print(json.dumps(rec), flush=True)
    write_breadth(rows, os.cpu_count(), cpu_model(), out)


def write_breadth(rows, nproc, model, path):
    """The breadth table (markdown, with a machine-readable JSON line that bench.py reads back)."""
    d = {"nproc": nproc, "cpu_model": model, "rtol": 1e-8,
         "note": "oracle (numpy/scipy FP64) on the host cores; direct = sparse LU of the bordered operator "
                 "(skipped at 512^2 and for SC, where it repeats another row); FGMRES = the oracle's FGMRES "
                 "with its V-cycle; setup = operator and hierarchy", "rows": rows}
    lines = ["# Oracle CPU baseline on configurations 0-3", "",
             "Command: `python bench.py --cpu-breadth` (run on the GPU box's host cores; each case in a fresh "
             "process, one thread = OMP/OpenBLAS/MKL limited to 1).", "",
             f"Host: {d['nproc']} cores, {d['cpu_model']}.", "",
             "| case | threads | set-up s | FGMRES s | iterations | direct s |", "|---|---|---:|---:|---:|---:|"]
    for r in rows:
        lines.append(f"| {r['case']} | {r['threads']} | {r.get('setup_s')} | {r.get('fgmres_s')} | "
                     f"{r.get('iterations')} | {r.get('direct_s')} |")
    lines += ["", "Machine-readable copy (read by bench.py into `cpu_baseline.breadth`):", "", json.dumps(d), ""]
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    open(path, "w").write("\n".join(lines))
    print(f"wrote {path}")


# ------------------------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle as the reference arm: rank 0 alone, on the host cores (one thread), each step a
    bounded sample of the headline workload (one FGMRES iteration's V-cycle and operator application),
    with the oracle's set-up and gradient timed once; value = ms per differentiated solve, scaled by
    HEAD_ITERATIONS."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import adjoint, multigrid, system
    from paper_1612_02208_gb300 import inputs
    prob = inputs.disk_and_ellipse_re(N_HEAD)
    t0 = time.perf_counter()
    L = system.operator_of(prob)
    b = system.rhs(prob)
    Hh = multigrid.Hierarchy(prob, smoother="sc", krylov=True)
    t_setup = time.perf_counter() - t0
    z = b
    for _ in range(max(args.warmup, 0)):
        z = Hh.vcycle(b)
        L @ z
    per = []
    t = time.perf_counter()
    for _ in range(args.steps):
        ts = time.perf_counter()
        z = Hh.vcycle(b)
        L @ z
        per.append(time.perf_counter() - ts)
    wall = time.perf_counter() - t
    tg = time.perf_counter()
    adjoint.gradients(prob, z, z)
    t_grad = time.perf_counter() - tg
    t_iter = float(np.mean(per))
    value = (t_setup + t_grad + (HEAD_ITERATIONS[0] + HEAD_ITERATIONS[1]) * t_iter) * 1e3
    threads = os.environ.get("OMP_NUM_THREADS", "default")
    sample = (f"{args.steps} steps of one oracle FGMRES iteration's V-cycle + operator application on the headline "
              f"workload ({t_iter:.2f} s each), oracle set-up {t_setup:.1f} s and gradient formula {t_grad:.1f} s "
              f"timed once; scaled to {HEAD_ITERATIONS[0]} + {HEAD_ITERATIONS[1]} iterations")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms/step", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(value, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_HEAD, "markers": prob.structure.M, "springs": prob.structure.E,
                   "kappa": 1e4, "rtol": 1e-8, "max_it": 100, "parallelism": "rank 0 only (CPU)"},
        "cpu_baseline": {"kind": "oracle", "cores": 1 if threads == "1" else os.cpu_count(), "value": round(value, 1),
                         "unit": "ms/step", "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": round(value, 1), "unit": "ms/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(wall, 2),
    }
    print(json.dumps(line), flush=True)


def run_profile_vcycle(which):
    """Two V-cycles (FP32 unless stated) with a one-vector FGMRES basis, so that the device holds little
    memory: the
    case ncu captures of the V-cycle kernels use.  'headline': the headline workload and smoother;
    'large': the 4096^2 thin ellipse (rho = 1, kappa = 1e4) with Vanka, the roofline leg's V-cycle;
    'large64': that body on 2048^2 with the FP64 V-cycle; 'large2k': that body on 2048^2 in FP32;
    'ras16': the 128^2 thick annulus (Stokes, gamma = 50) with the paper's 16 x 16 boxes of overlap 4;
    'ras8o2': the 2048^2 grid without a structure
    (rho = 1), RAS with 8 x 8 boxes of overlap 2, their correction on the tensor cores."""
    import torch
    from paper_1612_02208_gb300 import inputs, sib
    fp32 = 1
    if which == "headline":
        prob = inputs.disk_and_ellipse_re(N_HEAD)
        opts = dict(smoother=sib.SMOOTHER_SC, smooth_krylov=1)
    elif which == "large64":   # the FP64 V-cycle (FP64 pipe), on 2048^2 to keep the device memory small
        prob = inputs.thin_ellipse_re(LARGE_N // 2, kappa=1e4, seed=2)
        opts = dict(smoother=sib.SMOOTHER_VANKA)
        fp32 = 0
    elif which == "large2k":   # the roofline leg's body on 2048^2, FP32, for full captures of its kernels
        prob = inputs.thin_ellipse_re(LARGE_N // 2, kappa=1e4, seed=2)
        opts = dict(smoother=sib.SMOOTHER_VANKA)
    elif which == "ras16":   # the paper's 16 x 16 boxes with overlap 4: the 128^2 thick annulus, Stokes, gamma = 50
        prob = inputs.paper_problem("annulus", 128, 50.0)
        opts = dict(smoother=sib.SMOOTHER_RAS, box=HUGE_BOX[0], box_overlap=HUGE_BOX[1], ras_tc=1)
    elif which == "ras8o2":   # no structure: every box takes the tensor-core correction, about 3 GB on the device
        prob = inputs.no_structure(LARGE_N // 2, rho=1.0, seed=2)
        opts = dict(smoother=sib.SMOOTHER_RAS, box=WIDE_BOX[0], box_overlap=WIDE_BOX[1], ras_tc=1)
    else:
        prob = inputs.thin_ellipse_re(LARGE_N, kappa=1e4, seed=2)
        opts = dict(smoother=sib.SMOOTHER_VANKA)
    N = prob.N
    dev = torch.device("cuda")
    S = sib.solver_for(prob, vcycle_fp32=fp32, omega=-1.0, restart=1, max_it=1, **opts)
    b = torch.as_tensor(np.random.default_rng(5).standard_normal(3 * N * N), device=dev)
    b = b.float() if fp32 else b
    z = torch.empty_like(b)
    S.vcycle(b, z)   # the graph is captured outside the range
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("vcycle")
    for _ in range(2):
        S.vcycle(b, z)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"profile_vcycle": prob.name, "device_bytes": S.device_bytes, "launches": S.launch_count,
                      "z_norm": float(z.double().norm())}))
    S.close()


def run_profile_setup():
    """The headline's per-step set-up (set_structure + setup: binning, windows, patch factors, SC
    eigenvalue estimates, coarsest pseudo-inverse), twice inside an NVTX range "setup" after one
    outside it, each timed by CUDA events: the case the set-up's launch list uses."""
    import torch
    from paper_1612_02208_gb300 import sib
    dev = torch.device("cuda")
    H = Headline(sib, torch, dev)
    stream = torch.cuda.current_stream()
    H.S.set_structure(H.X, H.E, H.kap)
    H.S.setup()
    torch.cuda.synchronize()
    ms = []
    torch.cuda.nvtx.range_push("setup")
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        H.S.set_structure(H.X, H.E, H.kap)
        H.S.setup()
        e1.record(stream)
        e1.synchronize()
        ms.append(round(e0.elapsed_time(e1), 3))
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"profile_setup": H.prob.name, "setup_ms": ms, "launches": H.S.launch_count}))
    H.S.close()


def run_profile_solve():
    """One FGMRES solve (Vanka, kappa = 1e2, FP32 V-cycle) of the 128^2 disk without CUDA graphs."""
    import torch
    from paper_1612_02208_gb300 import inputs, sib
    prob = inputs.disk_stokes(128, kappa=1e2, seed=1)
    S = sib.solver_for(prob, use_graphs=0)
    g = torch.as_tensor(prob.g, device="cuda")
    S.solve(g)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("solve")
    w = S.solve(g)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"profile_solve": prob.name, "iterations": S.stats.iterations, "w_norm": float(w.norm())}))
    S.close()


def main(argv=None):
    args = parse_args(argv)
    if args.profile_vcycle:
        run_profile_vcycle(args.profile_vcycle)
    elif args.profile_setup:
        run_profile_setup()
    elif args.profile_solve:
        run_profile_solve()
    elif args.cpu_breadth:
        run_cpu_breadth(args.breadth_out)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()

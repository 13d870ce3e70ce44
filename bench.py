#!/usr/bin/env python
"""Benchmark of the Stokes-IB solve: FP64 flexible GMRES preconditioned by an FP32 multigrid
V-cycle, to a 1e-8 relative residual, on the thick-disk workload.

Workload (one step): periodic 128 x 128 MAC grid, Stokes flow (rho = 0, mu = 1, dt = 1e-2), an
elastic disk of radius 0.25 made of concentric marker rings at half-cell spacing (13,070 markers,
26,138 zero-rest-length springs), seeded N(0,1) forcing; the stiffness is swept over
kappa in {1e0, 1e2, 1e4, 1e6} for both the additive-Vanka and the Schur-complement smoother.
A step is those 8 solves, each with its set-up (stiffness, Galerkin coarse operators, coarsest
pseudo-inverse, eigenvalue estimates) and its FGMRES solve (cap 100 iterations).

Output: one JSON line (rank 0).  `value` is device time per solve in milliseconds over the
whole job (all ranks; replicas), `e2e` the same through the host-buffer C call.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
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

import numpy as np  # noqa: E402

METRIC = "Stokes-IB solve time to 1e-8 rel resid; V-cycle Mdof/s & %HBM; FP32 vs FP64 MG"
KAPPAS = [1e0, 1e2, 1e4, 1e6]
SMOOTHERS = ["vanka", "sc"]
N_GRID = 128
WORKLOAD = "disk_stokes_N128_kappa_sweep"
LARGE_N = 4096
L2_BYTES = 129 * 2 ** 20
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")
KERNEL_SOURCE = os.path.join(ROOT, "paper_1612_02208_gb300", "csrc", "kernels_grid.cu")


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-large", action="store_true", help="skip the large-grid V-cycle roofline")
    p.add_argument("--no-paper", action="store_true", help="skip the paper-workload iteration table")
    p.add_argument("--kappas", default=",".join(str(k) for k in KAPPAS),
                   help="comma-separated stiffness values of the sweep (default: the full workload)")
    p.add_argument("--smoothers", default=",".join(SMOOTHERS), help="comma-separated subset of vanka,sc")
    p.add_argument("--large-n", type=int, default=LARGE_N, help="grid of the large-grid V-cycle roofline")
    a = p.parse_args(argv)
    KAPPAS[:] = [float(x) for x in a.kappas.split(",")]
    SMOOTHERS[:] = [x for x in a.smoothers.split(",")]
    return a


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


def job_ms_per_solve(max_time_ms: float, solves_per_rank: int, world: int) -> float:
    """Whole-job time per solve: the slowest rank's time over the solves all ranks completed."""
    return max_time_ms / float(solves_per_rank * world)


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
            self.path = tempfile.mktemp(suffix=".csv")
            self.fh = open(self.path, "w")
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
        rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
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


def source_hash():
    return hashlib.sha256(open(KERNEL_SOURCE, "rb").read()).hexdigest()[:12]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    h = source_hash()
    for line in open(TRAFFIC_FILE):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == workload and f[3] == h:
            return float(f[2])
    return None


# ------------------------------------------------------------------------------------ native arm
def make_problem():
    from paper_1612_02208_gb300 import inputs
    return inputs.disk_stokes(N_GRID, kappa=1.0, seed=1)


def native_step(S, g, w, kap_dev, sib, records=None, vcycle_fp32=1, smooth_krylov=0):
    for sm in SMOOTHERS:
        S.set_options(smoother=sib.SMOOTHER_SC if sm == "sc" else sib.SMOOTHER_VANKA, vcycle_fp32=vcycle_fp32,
                      omega=-1.0, smooth_krylov=smooth_krylov)
        for kap in KAPPAS:
            S.set_stiffness(kap_dev[kap])
            S.setup()
            S.solve(g, w, allow_unconverged=True)
            if records is not None:
                d = S.stats.as_dict()
                records.append(dict(smoother=sm, kappa=kap, iterations=d["iterations"], converged=d["converged"],
                                    rel_residual=d["rel_residual"], setup_ms=round(d["setup_ms"], 4),
                                    solve_ms=round(d["solve_ms"], 4)))


def sc_gauss_seidel_cases(S, g, w, kap_dev, sib, torch, stream, smooth_krylov):
    """The step's SC solves (kappa sweep, FP32 V-cycle) with symmetric red-black Gauss-Seidel
    preconditioning both Chebyshev iterations (Sec. 3.3, SC smoothing), damped or wrapped."""
    S.set_options(smoother=sib.SMOOTHER_SC, vcycle_fp32=1, omega=-1.0, smooth_krylov=smooth_krylov,
                  sc_relax=sib.RELAX_SGS)
    records = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for kap in KAPPAS:
        S.set_stiffness(kap_dev[kap])
        S.setup()
        S.solve(g, w, allow_unconverged=True)
        d = S.stats.as_dict()
        records.append(dict(kappa=kap, iterations=d["iterations"], converged=d["converged"],
                            rel_residual=d["rel_residual"], setup_ms=round(d["setup_ms"], 4),
                            solve_ms=round(d["solve_ms"], 4)))
    e1.record(stream)
    e1.synchronize()
    S.set_options(sc_relax=sib.RELAX_JACOBI, smooth_krylov=0)
    return {"ms_per_solve": round(e0.elapsed_time(e1) / len(KAPPAS), 4), "cases": records}


def box_ras_cases(S, g, w, kap_dev, sib, torch, stream, box=4, overlap=1):
    """The step's kappa sweep with the box RAS smoother (Sec. 3.3, Alg. 2 with box x box subdomains and
    `overlap` cells of overlap; FP32 V-cycle, undamped)."""
    S.set_options(smoother=sib.SMOOTHER_RAS, vcycle_fp32=1, omega=-1.0, smooth_krylov=0, box=box,
                  box_overlap=overlap)
    records = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for kap in KAPPAS:
        S.set_stiffness(kap_dev[kap])
        S.setup()
        S.solve(g, w, allow_unconverged=True)
        d = S.stats.as_dict()
        records.append(dict(kappa=kap, iterations=d["iterations"], converged=d["converged"],
                            rel_residual=d["rel_residual"], setup_ms=round(d["setup_ms"], 4),
                            solve_ms=round(d["solve_ms"], 4)))
    e1.record(stream)
    e1.synchronize()
    S.set_options(smoother=sib.SMOOTHER_VANKA, box=4, box_overlap=1)
    return {"box": box, "overlap": overlap, "ms_per_solve": round(e0.elapsed_time(e1) / len(KAPPAS), 4),
            "cases": records}


WIDE_BOX = (8, 2)   # the paper's 8 x 8 boxes with overlap 2 (Sec. 5.1.1, 5.2.1)


def wide_boxes_accepted(sib):
    """Whether the library's options accept the paper's 8 x 8 boxes with overlap 2."""
    S = sib.Solver(32)
    try:
        S.set_options(smoother=sib.SMOOTHER_RAS, box=WIDE_BOX[0], box_overlap=WIDE_BOX[1])
        return True
    except sib.SibError:
        return False
    finally:
        S.close()


def paper_workloads(sib, torch, dev):
    """The paper's thick annulus and thin circle (Sec. 5.1, 5.2) in the periodic box: one linear solve
    each (dt = 0.32 h, g = 0, tolerance 1e-12, at most 100 iterations, FP32 V-cycle), over gamma,
    Stokes and mu = 0.01, and the smoothers; plus the annulus under grid refinement."""
    from paper_1612_02208_gb300 import inputs
    smoothers = {"vanka": dict(smoother=sib.SMOOTHER_VANKA), "sc": dict(smoother=sib.SMOOTHER_SC),
                 "ras4o1": dict(smoother=sib.SMOOTHER_RAS, box=4, box_overlap=1),
                 "ras2o2": dict(smoother=sib.SMOOTHER_RAS, box=2, box_overlap=2)}
    if wide_boxes_accepted(sib):
        smoothers["ras8o2"] = dict(smoother=sib.SMOOTHER_RAS, box=WIDE_BOX[0], box_overlap=WIDE_BOX[1])
    runs = [(kind, 128, gamma, mu, sm) for kind in ("annulus", "circle") for mu in (None, 0.01)
            for gamma in (5.0, 50.0, 500.0) for sm in smoothers]
    runs += [("annulus", N, gamma, None, sm) for N in (64, 256) for gamma in (5.0, 500.0) for sm in ("vanka", "ras4o1")]
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
            "boundary": "periodic (the paper's lid-driven cavity walls are not modelled)", "cases": cases}


def cavity_accepted(sib):
    """Whether the library's options accept the lid-driven cavity domain."""
    S = sib.Solver(32)
    try:
        S.set_options(domain=sib.DOMAIN_CAVITY)
        return True
    except sib.SibError:
        return False
    finally:
        S.close()


def cavity_workloads(sib, torch, dev):
    """The paper's lid-driven cavity (Sec. 5: no-slip walls, regularised lid) with its thick annulus and
    thin circle, Stokes flow, one linear solve each (dt = 0.32 h, g = 0: the lid and the elastic force
    of the initial configuration drive the flow; tolerance 1e-12, at most 100 iterations, FP32 V-cycle,
    Vanka), over gamma."""
    if not cavity_accepted(sib):
        return {"unavailable": "the options do not accept the cavity domain"}
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


def e2e_step(S, g_host, w_host, kap_host, kap_dev, sib, torch):
    """Through the host-buffer call: stiffness uploaded from pinned memory, g in, w out."""
    for sm in SMOOTHERS:
        S.set_options(smoother=sib.SMOOTHER_SC if sm == "sc" else sib.SMOOTHER_VANKA, vcycle_fp32=1, omega=-1.0)
        for kap in KAPPAS:
            kap_dev[kap].copy_(kap_host[kap], non_blocking=True)
            S.set_stiffness(kap_dev[kap])
            S.setup()
            S.solve_host(g_host, w_host, allow_unconverged=True)


def large_vcycle(sib, torch, reps=20, N=None):
    """V-cycle throughput and the Vanka kernel's roofline on a grid whose working set exceeds L2
    (4096^2: one FP32 sweep moves 600 MB), rho = 1, mu = 1e-2, dt = 1e-3, thin ellipse,
    kappa = 1e4, FP32 V-cycle."""
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
    torch.cuda.nvtx.range_push("vcycles")
    for _ in range(3):
        S.vcycle(b, z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        S.vcycle(b, z)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    t_v = e0.elapsed_time(e1) / reps
    lmax = S.num_levels - 1
    out = {"workload": f"thin_ellipse_re_N{LARGE}_kappa1e4", "N": LARGE, "vcycle_ms": round(t_v, 4),
           "vcycle_mdofs": round(n3 / (t_v * 1e-3) / 1e6, 1), "kernels": {}}
    for name in ("vanka", "residual", "restrict", "prolong"):
        torch.cuda.nvtx.range_push("roofline_large_" + name)
        ms, by = S.time_kernel(name, lmax, True, reps=20)
        torch.cuda.nvtx.range_pop()
        out["kernels"][name] = {"ms": round(ms, 5), "bytes": by, "gbs": round(by / (ms * 1e-3) / 1e9, 1)}
    # the box RAS smoother on the same grid: V-cycle and correction kernel, 4 x 4 boxes with overlap 1
    # and, where the options accept them, the paper's 8 x 8 boxes with overlap 2
    shapes = [((4, 1), "ras")] + ([(WIDE_BOX, "ras8o2")] if wide_boxes_accepted(sib) else [])
    for (bx, ov), key in shapes:
        S.set_options(smoother=sib.SMOOTHER_RAS, box=bx, box_overlap=ov, omega=-1.0)
        S.setup()
        for _ in range(3):
            S.vcycle(b, z)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("vcycles_" + key)
        e0.record()
        for _ in range(reps):
            S.vcycle(b, z)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        out["vcycle_ms_" + key] = round(e0.elapsed_time(e1) / reps, 4)
        torch.cuda.nvtx.range_push("roofline_large_" + key)
        ms, by = S.time_kernel("ras", lmax, True, reps=20)
        torch.cuda.nvtx.range_pop()
        out["kernels"][key] = {"ms": round(ms, 5), "bytes": by, "gbs": round(by / (ms * 1e-3) / 1e9, 1)}
        # the correction is a dense product: 2 ne flops per owned dof, ne = 3 e^2 + 2 e, e = b + 2 o
        e = bx + 2 * ov
        flops = 2.0 * (3 * e * e + 2 * e) * 3.0 * LARGE * LARGE
        out["kernels"][key]["tflops"] = round(flops / (ms * 1e-3) / 1e12, 2)
    S.close()
    return out


def time_loop_leg(sib, torch, prob, dev, steps=5):
    """The semi-implicit time loop on the benchmark disk (Vanka, kappa = 1e2): every step sets the
    structure at X^n, sets up, solves to 1e-8 and moves the markers, X^{n+1} = X^n + dt J^n u^{n+1}.
    Timed by CUDA events around the loop (the set-up's host synchronisations included)."""
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


def run_native(args):
    import torch
    from paper_1612_02208_gb300 import sib

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    rank, world = dist_init("nccl")
    dev = torch.device("cuda", local)
    prob = make_problem()
    st = prob.structure
    S = sib.Solver(prob.N)
    S.set_fluid(prob.rho, prob.mu, prob.dt)
    X = torch.as_tensor(st.X, device=dev)
    Ed = torch.as_tensor(st.edges, device=dev)
    S.set_structure(X, Ed, torch.as_tensor(st.kappa, device=dev))
    kap_dev = {k: torch.full((st.E,), k, dtype=torch.float64, device=dev) for k in KAPPAS}
    g = torch.as_tensor(prob.g, device=dev)
    w = torch.empty_like(g)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    for _ in range(max(args.warmup, 0)):
        native_step(S, g, w, kap_dev, sib)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    dist_barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("timed_steps")
    launches0 = S.launch_count
    records = []
    step_ms = []
    t_wall = time.perf_counter()
    stream = torch.cuda.current_stream()
    for k in range(args.steps):
        flush.fill_(float(k))                     # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        native_step(S, g, w, kap_dev, sib, records if k == 0 else None)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dist_barrier()
    wall = time.perf_counter() - t_wall
    launches = S.launch_count - launches0
    clk = clocks.stop()

    total_ms = float(sum(step_ms))
    solves = len(SMOOTHERS) * len(KAPPAS)
    max_total = dist_max(total_ms, dev)
    value = job_ms_per_solve(max_total, solves * args.steps, world)

    # dominant kernel of the step, timed live on the benchmark's own context and stream
    lmax = S.num_levels - 1
    S.set_options(smoother=sib.SMOOTHER_VANKA, omega=-1.0)
    S.set_stiffness(torch.full((st.E,), 1e2, dtype=torch.float64, device=dev))
    S.setup()
    torch.cuda.nvtx.range_push("roofline_vanka")
    dom_ms, dom_bytes = S.time_kernel("vanka", lmax, True, reps=50)
    torch.cuda.nvtx.range_pop()
    peak, peak_kind = measured_peaks()
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_vanka<float> (finest level)", "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": recorded_traffic("k_vanka_f32", WORKLOAD), "bytes_per_launch": dom_bytes,
                "launch_ms": round(dom_ms, 5), "peak_source": peak_kind,
                "note": "working set fits in L2 at N=128; see vcycle_large for the HBM-bound size"}

    # FP64 V-cycle for the same step (context: FP32 vs FP64 multigrid)
    fp64_records = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    flush.fill_(0.5)
    e0.record(stream)
    native_step(S, g, w, kap_dev, sib, fp64_records, vcycle_fp32=0)
    e1.record(stream)
    e1.synchronize()
    fp64_ms = e0.elapsed_time(e1) / solves

    # the paper's smoothing form (Sec. 3.3): every smoothing stage is FGMRES(nu) preconditioned by
    # one undamped basic sweep, on the same step
    kry_records = []
    flush.fill_(0.25)
    e0.record(stream)
    native_step(S, g, w, kap_dev, sib, kry_records, smooth_krylov=1)
    e1.record(stream)
    e1.synchronize()
    kry_ms = e0.elapsed_time(e1) / solves
    S.set_options(smooth_krylov=0)

    # SC with Gauss-Seidel (the paper's relaxation) instead of Jacobi inside its Chebyshev iterations
    sc_gs = {"damped": sc_gauss_seidel_cases(S, g, w, kap_dev, sib, torch, stream, 0),
             "wrapped": sc_gauss_seidel_cases(S, g, w, kap_dev, sib, torch, stream, 1)}
    # the paper's box Vanka smoother: restricted additive Schwarz over 4 x 4 and 2 x 2 boxes, overlap 1
    ras = [box_ras_cases(S, g, w, kap_dev, sib, torch, stream, 4, 1),
           box_ras_cases(S, g, w, kap_dev, sib, torch, stream, 2, 1)]
    if wide_boxes_accepted(sib):
        ras.append(box_ras_cases(S, g, w, kap_dev, sib, torch, stream, *WIDE_BOX))
    else:
        ras.append({"box": WIDE_BOX[0], "overlap": WIDE_BOX[1],
                    "unavailable": "the options accept subdomains up to 6 cells wide"})
    paper = paper_workloads(sib, torch, dev) if not args.no_paper else None
    cav = cavity_workloads(sib, torch, dev) if not args.no_paper else None

    # end to end through the host-buffer C call, pinned host memory
    g_host = torch.as_tensor(prob.g).pin_memory().numpy()
    w_host = torch.empty(g.numel(), dtype=torch.float64).pin_memory().numpy()
    kap_host = {k: torch.full((st.E,), k, dtype=torch.float64).pin_memory() for k in KAPPAS}
    e2e_step(S, g_host, w_host, kap_host, kap_dev, sib, torch)
    torch.cuda.synchronize()
    dist_barrier()
    t = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        e2e_step(S, g_host, w_host, kap_host, kap_dev, sib, torch)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t) * 1e3
    e2e_value = job_ms_per_solve(dist_max(e2e_ms, dev), solves * e2e_steps, world)
    n3 = 3 * prob.N * prob.N
    e2e = {"value": round(e2e_value, 4), "unit": "ms/solve", "h2d_bytes_per_step": solves * (8 * n3 + 8 * st.E),
           "d2h_bytes_per_step": solves * 8 * n3}

    tloop = time_loop_leg(sib, torch, prob, dev)

    large = None
    if not args.no_large:
        torch.cuda.nvtx.range_push("vcycle_large")
        large = large_vcycle(sib, torch, N=args.large_n)
        torch.cuda.nvtx.range_pop()
        large["roofline_vanka"] = {"achieved": large["kernels"]["vanka"]["gbs"], "peak": peak,
                                   "frac": round(large["kernels"]["vanka"]["gbs"] / peak, 4),
                                   "traffic": recorded_traffic("k_vanka_f32", large["workload"])}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ms, cases = oracle_sweep()
        cpu = {"value": round(ms, 2), "unit": "ms/solve", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one full step: the 8 solves of the kappa x smoother sweep, numpy/scipy FP64, "
                         "set-up included", "iterations": [c["iterations"] for c in cases]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "ms/solve", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(max_total / args.steps, 4), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": prob.N, "markers": st.M, "springs": st.E,
                       "kappa": KAPPAS, "smoothers": SMOOTHERS, "vcycle": "fp32, coarsest fp64",
                       "krylov": "fp64 FGMRES(100), CGS2", "rtol": 1e-8, "max_it": 100,
                       "parallelism": f"replicas x{world}", "l2": "flushed between timed steps",
                       "timing": "CUDA events per step on the launching stream"},
            "cases": records, "fp64_vcycle": {"ms_per_solve": round(fp64_ms, 4), "cases": fp64_records},
            "krylov_smoothing": {"ms_per_solve": round(kry_ms, 4), "cases": kry_records},
            "sc_gauss_seidel": sc_gs,
            "box_ras": ras,
            "paper_workloads": paper, "cavity_workloads": cav,
            "roofline": roofline, "time_loop": tloop, "vcycle_large": large, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk, "wall_s": round(wall, 3),
        }
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------ reference arm
def oracle_sweep():
    """The oracle (FP64 numpy/scipy) on one full step of the workload; returns (ms/solve, cases)."""
    from oracle import krylov, multigrid, system
    prob = make_problem()
    cases = []
    t0 = time.perf_counter()
    for sm in SMOOTHERS:
        for kap in KAPPAS:
            prob.structure.kappa[:] = kap
            L = system.operator_of(prob)
            b = system.rhs(prob)
            H = multigrid.Hierarchy(prob, smoother=sm)
            x, its, hist, conv = krylov.fgmres(lambda z: L @ z, H.vcycle, b, rtol=1e-8, max_it=100,
                                               project=lambda z: system.project(z, prob.N, prob.rho))
            cases.append(dict(smoother=sm, kappa=kap, iterations=its, converged=bool(conv)))
    ms = (time.perf_counter() - t0) * 1e3 / len(cases)
    return ms, cases


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(max(args.warmup, 0)):
        oracle_sweep()
    per = []
    cases = None
    t = time.perf_counter()
    for _ in range(args.steps):
        ms, cases = oracle_sweep()
        per.append(ms)
    wall = time.perf_counter() - t
    value = float(np.mean(per))
    solves = len(SMOOTHERS) * len(KAPPAS)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": "ms/solve", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(value * solves, 2),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_GRID, "kappa": KAPPAS, "smoothers": SMOOTHERS, "rtol": 1e-8,
                   "max_it": 100, "parallelism": "rank 0 only (CPU)"},
        "cases": cases,
        "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": round(value, 2), "unit": "ms/solve",
                         "sample": f"{args.steps} full steps of the workload (8 solves each), set-up included"},
        "e2e": {"value": round(value, 2), "unit": "ms/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(wall, 2),
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()

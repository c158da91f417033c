#!/usr/bin/env python3
"""Benchmark: time steps/s of the optimized Schwarz time stepper on one GB300.

Default workload (nls_well): NLS with a Gaussian well and focusing cubic term on (-32,32)^2,
1024 x 1024 cells, 16 x-strips, preconditioned Schwarz (eq. algo_pd) with Robin p = 2,
dt = 0.005, interface residual 1e-8.  The chosen form (FP32 inner Krylov, FP64 residuals and
interface) is timed against the plain FP64 path on the same GPU.

One "step" is one time step of eq. (CNS): every Schwarz iteration, strip solve, flux update
and preconditioned update of that step.  Inputs are resident in HBM; L2 is flushed (a 512 MB
write) before every timed step; each step is timed with CUDA events on the library's stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload nls_well|nls_small|gpe_trap|gpe_batch|learned_guess]

Under torchrun (N > 1) every rank runs an independent replica (the path has no cross-GPU
exchange on one node here), the slowest rank's time counts, and value = N*K / time.

Roofline of the strip solver (the dominant kernel): algorithmic bytes per Krylov iteration of
a strip are 68 B/node in FP32 (136 B/node in FP64): one complex stencil apply (read x and c,
write y: 8 + 4 + 8 B) plus six complex vector streams; the nonlinear residual applies in
between are counted separately at 40 B/node (the FP64 stencil).  achieved = bytes x nodes per
strip x strip-Krylov iterations / strip-solver time, against the measured HBM copy bandwidth.

The oracle baselines run the FP64 CPU oracle as it stands, its strip solves spread over the
host cores by worker processes (one strip per task, like one MPI rank per strip), with the exact
P^{-1} on the cosine modes for the preconditioned algorithm.
"""
import argparse
import copy
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time steps/s and stencil GB/s at 1e-8 interface residual, chosen vs plain FP64"

# algorithmic bytes per node: one Krylov iteration of a strip (stencil + six vector streams),
# and one FP64 stencil apply of the nonlinear residual
KRYLOV_BYTES = {"fp32": 68.0, "fp64": 136.0}
RESIDUAL_BYTES = 40.0

# DRAM traffic of the strip solver per launch (dram__bytes_read.sum + dram__bytes_write.sum from one
# ncu capture, the mean over every strip-solver launch of
#     python bench.py [--workload W] --steps 5 --warmup 3 --no-fp64 --no-cpu --no-extra
# for nls_well, --steps 3 for gpe_trap) and the hash of the kernel sources it was measured on; a
# figure is reported only while those sources are unchanged (null once the kernel changed).
KERNEL_SOURCES = ["strip_solver.cu", "common.cuh", "dw.cuh", "kernels.h"]
STRIP_TRAFFIC = {"nls_well": (47.51e6, "ada2ee9a76d08914"), "gpe_trap": (1979.2e6, "ada2ee9a76d08914")}


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1603_05110_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload):
    t = STRIP_TRAFFIC.get(workload)
    if t is None:
        return None, "no ncu capture of this workload"
    try:
        same = kernel_sources_hash() == t[1]
    except OSError:
        same = False
    if not same:
        return None, "the kernel sources changed since the ncu capture"
    return t[0], "ncu: mean DRAM bytes (read + write) per strip-solver launch of this workload"

def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: the workload's run length, nls_well 200; gpe_batch 3)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nls_well")
    ap.add_argument("--p", type=float, default=None, help="Robin p (default: the workload's)")
    ap.add_argument("--tc", default=None, choices=["robin", "pade"],
                    help="transmission operator (default: the workload's, else Robin)")
    ap.add_argument("--pade-m", type=int, default=None, help="Pade order (default: the workload's, else 4)")
    ap.add_argument("--algorithm", default="workload", choices=["workload", "classical", "preconditioned"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="plain FP64 steps, from the chosen form's post-warm-up state (default: --steps)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--residual", default="dw", choices=["fp64", "dw"],
                    help="nonlinear residual of the chosen form: FP64, or double-word on the FP32 pipe")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--batch-form", default="chosen", choices=["chosen", "classical"],
                    help="gpe_batch: preconditioned + double-word residual (chosen) or classical + FP32 inner")
    ap.add_argument("--no-extra", action="store_true",
                    help="nls_well: skip the gpe_trap and gpe_batch lines nested under 'configs'")
    ap.add_argument("--learn-n", type=int, default=1024, help="learned_guess: cells per direction")
    ap.add_argument("--learn-strips", type=int, default=32)
    ap.add_argument("--learn-train", type=int, default=2000, help="learned_guess: training steps generated")
    ap.add_argument("--learn-traj", type=int, default=4, help="learned_guess: training trajectories (one beta each)")
    ap.add_argument("--learn-eval", type=int, default=500, help="learned_guess: held-out steps")
    ap.add_argument("--learn-epochs", type=int, default=3)
    ap.add_argument("--max-schwarz", type=int, default=5000)
    ap.add_argument("--cpu-budget", type=float, default=30.0,
                    help="seconds of oracle work for the cpu_baseline sample")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds of timed oracle steps in the reference arm")
    args = ap.parse_args(argv)
    from paper_1603_05110_gb300 import workloads as wl
    w = wl.WORKLOADS.get(args.workload)
    extra = w.extra if w is not None else {}
    if args.steps is None:
        args.steps = w.steps if w is not None else 3
    if args.tc is None:
        args.tc = extra.get("tc", "robin")
    if args.pade_m is None:
        args.pade_m = extra.get("pade_m", 4)
    return args


def robin_p(w, args):
    return args.p if getattr(args, "p", None) is not None else w.p


def algorithm_of(w, args):
    a = getattr(args, "algorithm", "workload")
    return w.algorithm if a == "workload" else a


def solver_params(w, args, precision, psolve=None, adapt=0.01):
    from paper_1603_05110_gb300 import binding
    pade = getattr(args, "tc", "robin") == "pade"
    return dict(psolve=binding.PSOLVE_MODAL if psolve is None else psolve, nl_adapt=adapt,
                xl=w.xl, xr=w.xr, yb=w.yb, yu=w.yu, nx=w.nx, ny=w.ny, n_strips=w.n_strips, dt=w.dt, lap=w.lap,
                kappa=w.kappa, p=robin_p(w, args), tol=args.tol, nl_tol=1e-11, inner_tol=1e-4,
                max_inner=4000, max_schwarz=400, gmres_tol=1e-6, gmres_restart=30, gmres_max=300,
                algorithm=binding.PRECONDITIONED if algorithm_of(w, args) == "preconditioned" else binding.CLASSICAL,
                tc=binding.TC_PADE if pade else binding.TC_ROBIN, pade_m=getattr(args, "pade_m", 4),
                precision=precision, guess=binding.GUESS_PREVIOUS, nl_relax=w.extra.get("relax", 1.0),
                omega_rot=w.extra.get("omega", 0.0))


def describe(w, args):
    return (f"{w.name}: {w.nx}x{w.ny} cells on ({w.xl:g},{w.xr:g})x({w.yb:g},{w.yu:g}), {w.n_strips} strips, "
            f"{algorithm_of(w, args)} Schwarz, "
            + (f"S_pade m={args.pade_m}" if getattr(args, "tc", "robin") == "pade" else f"Robin p={robin_p(w, args):g}")
            + f", dt={w.dt:g}, interface tol {args.tol:g}")


class Clocks:
    """nvidia-smi sampling during the timed region: started before it, waited for until its first
    sample is out (its start-up must not fall into the timed region), and only the samples
    written after that are read."""

    def __init__(self, index, ready_timeout=5.0):
        self.proc = None
        self.skip = 0
        fd, self.path = tempfile.mkstemp(prefix="ddnls_clocks_", suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        if self.proc is not None:
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < ready_timeout and self.proc.poll() is None:
                self.f.flush()
                try:
                    with open(self.path) as fh:
                        n = sum(1 for _ in fh)
                except OSError:
                    n = 0
                if n >= 1:
                    self.skip = n
                    break
                time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = open(self.path).read().splitlines()
        if len(lines) > self.skip:
            lines = lines[self.skip:]        # the samples of the timed region
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------- multi-rank helpers
def max_over_ranks(value, dist=None, device=None):
    """The largest value over all ranks (the slowest rank's time); the value itself at N = 1."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, slowest_ms):
    """Units all ranks processed (world replicas x steps) per second of the slowest rank."""
    return world * steps / (slowest_ms * 1e-3)


# ------------------------------------------------------------------------- oracle timing
def host_info():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model}


def oracle_problem(w, args, V=None):
    from oracle import nls
    return nls.Problem(xl=w.xl, xr=w.xr, yb=w.yb, yu=w.yu, nx=w.nx, ny=w.ny, dt=w.dt, V=w.V() if V is None else V,
                       kappa=w.kappa, lap=w.lap, p=robin_p(w, args),
                       tc="pade" if getattr(args, "tc", "robin") == "pade" else "robin", m=getattr(args, "pade_m", 4))


def oracle_steps(w, args, n_steps, budget_s, warm_steps=0, max_iter_first=None):
    """The oracle as it stands on the host cores: strip solves of each Schwarz iteration in worker
    processes, the exact P^{-1} on the cosine modes (preconditioned), strip fixed points to the
    chosen form's strip tolerance.  warm_steps untimed steps from u0 (zero guess), then up to
    n_steps timed steps from the previous step's converged interface vector, stopping once
    budget_s is spent.  max_iter_first: time only that many Schwarz iterations of the first step
    (a bounded sample of a step too long to run whole).  Returns a dict of what was timed."""
    from oracle import nls
    prob = oracle_problem(w, args)
    procs = max(1, min(os.cpu_count() or 1, w.n_strips))
    algorithm = algorithm_of(w, args)
    relax = w.extra.get("relax", 1.0)
    out = {"processes": procs, "steps": [], "iterations": [], "setup_s": 0.0}
    with nls.strip_pool(prob, w.n_strips, procs) as pool:
        st = nls.Strips(prob, w.n_strips, pool=pool)
        modal = None
        if algorithm == "preconditioned":
            t0 = time.perf_counter()
            modal = st.modal_blocks()
            out["setup_s"] = time.perf_counter() - t0
        u, g = w.u0(), None
        kw = dict(algorithm=algorithm, tol=args.tol, strips=st, psolve="modal", modal=modal, tol_fp=1e-11,
                  relax=relax)
        for _ in range(warm_steps):
            u, _, info = nls.schwarz_step(prob, w.n_strips, u, g0=g, **kw)
            g = info.g
        spent = 0.0
        for k in range(n_steps):
            t0 = time.perf_counter()
            if max_iter_first is not None and k == 0:
                u, _, info = nls.schwarz_step(prob, w.n_strips, u, g0=g, max_iter=max_iter_first, strict=False, **kw)
            else:
                u, _, info = nls.schwarz_step(prob, w.n_strips, u, g0=g, **kw)
            dt_s = time.perf_counter() - t0
            out["steps"].append(dt_s)
            out["iterations"].append(info.iterations)
            out["converged"] = info.converged
            g = info.g
            spent += dt_s
            if spent >= budget_s or not info.converged:
                break
    return out


def cpu_baseline_line(w, args, gpu_iters_per_step):
    """A bounded sample of the oracle on the same workload, scaled to steps/s."""
    hi = host_info()
    whole = w.nodes() <= 1.2e6 and w.n_strips <= 64
    if whole:
        r = oracle_steps(w, args, 1, args.cpu_budget)
        t, its = r["steps"][0], r["iterations"][0]
        value = 1.0 / t
        sample = (f"one whole oracle step: step 1 of {w.name} from u0 with the zero interface guess "
                  f"({its} Schwarz iterations, {w.n_strips} strip solves each over {r['processes']} worker "
                  f"processes, exact modal P^-1), {t:.1f} s; cosine-mode set-up {r['setup_s']:.2f} s not counted; "
                  f"host {hi['cpu']}, {hi['nproc']} cores")
    else:
        k = 1
        r = oracle_steps(w, args, 1, args.cpu_budget, max_iter_first=k)
        t, its = r["steps"][0], r["iterations"][0]
        value = 1.0 / (t / its * gpu_iters_per_step)
        sample = (f"the first {its} Schwarz iteration(s) of step 1 of {w.name} ({w.n_strips} strip solves each over "
                  f"{r['processes']} worker processes), {t:.1f} s, scaled to the {gpu_iters_per_step:.1f} Schwarz "
                  f"iterations per step this run measured on the GPU; host {hi['cpu']}, {hi['nproc']} cores")
    return {"value": value, "unit": "steps/s", "cores": r["processes"], "kind": "oracle", "sample": sample,
            "host": hi}


def run_reference(args, rank):
    """The oracle as it stands, on the host cores, timed on whole steps of the same workload."""
    from paper_1603_05110_gb300 import workloads as wl
    if rank != 0:
        return
    w = wl.WORKLOADS[args.workload]
    t_start = time.perf_counter()
    r = oracle_steps(w, args, max(1, args.steps), args.ref_budget, warm_steps=1)
    n = len(r["steps"])
    total = sum(r["steps"])
    value = n / total
    hi = host_info()
    sample = (f"{n} whole oracle steps (steps 2..{n + 1} of {w.name}, each from the previous step's converged "
              f"interface vector, {statistics.mean(r['iterations']):.1f} Schwarz iterations per step, "
              f"{w.n_strips} strip solves per iteration over {r['processes']} worker processes, exact modal "
              f"P^-1); step 1 from u0 untimed; cosine-mode set-up {r['setup_s']:.2f} s not counted; "
              f"host {hi['cpu']}, {hi['nproc']} cores")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": n, "warmup": 1, "ms_per_step": total / n * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(w, args)},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": r["processes"], "kind": "oracle",
                             "sample": sample, "host": hi},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "timed_region_s": total, "wall_s": time.perf_counter() - t_start,
            "note": f"--steps {args.steps} requested; the oracle times whole steps until {args.ref_budget:g} s "
                    f"of timed steps are spent"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- roofline
def strip_roofline(prof, stats, w, prec, peaks, peak_kind, nodes_per_strip=None):
    """The strip solver's achieved bandwidth from algorithmic bytes: KRYLOV_BYTES[prec] per node
    per strip-Krylov iteration, over the solver's CUDA-event time; the residual applies are listed
    apart at RESIDUAL_BYTES per node (one per correction plus the final check of each strip in each
    launch)."""
    nps = nodes_per_strip if nodes_per_strip is not None else (w.nx // w.n_strips + 1) * (w.ny + 1)
    launches = max(1, prof["strip_solve_launches"])
    kry = sum(s["krylov_iterations"] for s in stats)
    nl = sum(s["nl_iterations"] for s in stats)
    res_applies = nl + launches * w.n_strips
    t = prof["strip_solve_ms"] * 1e-3
    kb = KRYLOV_BYTES[prec] * nps * kry
    rb = RESIDUAL_BYTES * nps * res_applies
    out = {"kernel": f"strip_solve_kernel<{'float' if prec == 'fp32' else 'double'}>", "bound": "hbm",
           "achieved": kb / t / 1e9, "unit": "GB/s",
           "krylov_bytes_per_launch": kb / launches, "ms_per_launch": prof["strip_solve_ms"] / launches,
           "strip_krylov_iterations": kry, "residual_applies": res_applies,
           "achieved_with_residual": (kb + rb) / t / 1e9, "traffic": None,
           "note": f"{KRYLOV_BYTES[prec]:g} B/node per strip-Krylov iteration x {nps} nodes per strip x "
                   f"iterations / strip-solver time (CUDA events on the library stream); residual applies at "
                   f"{RESIDUAL_BYTES:g} B/node in achieved_with_residual"}
    if prec == "fp32":
        out["traffic"], out["traffic_source"] = measured_traffic(w.name)
    if peaks is not None:
        out.update(peak=peaks["hbm_gbs"], frac=out["achieved"] / peaks["hbm_gbs"], peak_source=f"{peak_kind} hbm_gbs")
    return out


# ---------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1603_05110_gb300 import binding, build, workloads as wl
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev) if "device_id" in dist.init_process_group.__code__.co_varnames \
            else dist.init_process_group("nccl")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = wl.WORKLOADS[args.workload]
    u0 = torch.from_numpy(w.u0()).to(dev)
    V = torch.from_numpy(w.V()).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed_steps(solver, k, profile=False):
        if profile:
            solver.set_profiling(True)
        ms, stats = [], []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats.append(solver.step(1))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        prof = solver.profile() if profile else None
        return ms, stats, prof

    # ---- chosen form: FP32 inner Krylov + FP64 (or double-word) residuals, FP64 interface
    CHOSEN = binding.FP32_DW if args.residual == "dw" else binding.FP32_INNER
    chosen = binding.Solver(solver_params(w, args, CHOSEN), u0, V, stream=stream)
    for _ in range(args.warmup):
        chosen.step(1)
    # the state after the warm-up: the timed steps, their profiled repeat and the end-to-end steps
    # all start from it, so the three cover the same stretch of the trajectory
    ntr = 2 * (w.n_strips - 1)
    u_w = torch.empty_like(u0)
    g_w = torch.empty(ntr, w.ny + 1, dtype=torch.complex128, device=dev) if ntr > 0 else None
    n_w = chosen.get_state(u_w, g_w)
    barrier()
    clocks = Clocks(local_rank)
    barrier()
    ms, stats, _ = timed_steps(chosen, args.steps)      # the headline: the library's profiling off
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(ms), dist, dev)
    value = whole_job_rate(world, args.steps, total_ms)
    iters = [s["last_schwarz_iterations"] for s in stats]
    # the same number of steps again with the library's profiling on (CUDA events around each
    # phase, each read back at once): the time split, the strip solver's kernel time for the
    # roofline and the launch count come from this repeat
    chosen.set_state(u_w, g_w, n_w)
    ms_p, stats_p, prof = timed_steps(chosen, args.steps, profile=True)
    chosen.set_profiling(False)
    kry = sum(s["krylov_iterations"] for s in stats_p)

    # ---- e2e through the C-ABI with host buffers (pinned): H2D of u_{n-1}, step, D2H of u_n
    uh_in = torch.empty(w.ny + 1, w.nx + 1, dtype=torch.complex128, pin_memory=True)
    uh_out = torch.empty_like(uh_in)
    chosen.set_state(u_w, g_w, n_w)
    uh_in.copy_(u_w)
    step_no = n_w
    e2e_ms = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        chosen.set_state(uh_in, None, step_no)
        chosen.step(1, uh_out)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        step_no += 1
        uh_in.copy_(uh_out)
    chosen.close()
    node_bytes = 16 * (w.nx + 1) * (w.ny + 1)

    # ---- plain FP64 on the same GPU, and the accuracy of the chosen form against it
    fp64 = None
    err = None
    if not args.no_fp64 and rank == 0:
        # the same steps as the chosen form's timed region: from its post-warm-up state
        k64 = args.fp64_steps if args.fp64_steps else args.steps
        plain = binding.Solver(solver_params(w, args, binding.FP64), u0, V, stream=stream)
        plain.step(1)
        plain.set_state(u_w, g_w, n_w)
        ms64, st64, _ = timed_steps(plain, k64)
        kp = min(k64, 10)
        plain.set_state(u_w, g_w, n_w)
        _, st64p, prof64 = timed_steps(plain, kp, profile=True)
        plain.close()
        fp64 = {"value": k64 / (sum(ms64) * 1e-3), "unit": "steps/s", "steps": k64,
                "ms_per_step": sum(ms64) / k64,
                "schwarz_iterations_per_step": statistics.mean(s["last_schwarz_iterations"] for s in st64),
                "strip_solve_gbs": strip_roofline(prof64, st64p, w, "fp64", None, None)["achieved"],
                "strip_solve_ms_per_step": prof64["strip_solve_ms"] / kp,
                "note": f"from the chosen form's post-warm-up state; strip figures from a profiled repeat of the first {kp} steps"}
        # the paper-literal path: FP64, L_h from unit solves, P x = y by GMRES (Robin only: the
        # library solves S_pade's preconditioned update by the modal solve)
        if args.tc == "robin" and algorithm_of(w, args) == "preconditioned":
            gm = binding.Solver(solver_params(w, args, binding.FP64, binding.PSOLVE_GMRES, adapt=0.0), u0, V,
                                stream=stream)
            gm.step(1)
            msg, stg, _ = timed_steps(gm, 2)
            gm.close()
            fp64["paper_literal_gmres"] = {"value": 2 / (sum(msg) * 1e-3), "unit": "steps/s",
                                           "ms_per_step": sum(msg) / 2,
                                           "gmres_iterations_per_step": statistics.mean(s["gmres_iterations"] for s in stg),
                                           "setup_ms": stg[0]["setup_ms"]}
        # same number of steps from u0 in both forms
        nchk = 3
        ua = torch.empty_like(u0)
        ub = torch.empty_like(u0)
        with binding.Solver(solver_params(w, args, CHOSEN), u0, V, stream=stream) as s:
            s.step(nchk, ua)
        with binding.Solver(solver_params(w, args, binding.FP64), u0, V, stream=stream) as s:
            s.step(nchk, ub)
        err = float(torch.linalg.vector_norm(ua - ub) / torch.linalg.vector_norm(ub))

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    dw_used = args.residual == "dw"
    peaks, peak_kind = measured_peaks()
    roofline = strip_roofline(prof, stats_p, w, "fp32", peaks, peak_kind)
    roofline["share_of_step"] = prof["strip_solve_ms"] / sum(ms_p)

    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline_line(w, args, statistics.mean(iters))

    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 inner Krylov + " + ("double-word f32x2" if dw_used else "f64") + " residual, f64 interface",
        "data": "synthetic",
        "config": {"workload": describe(w, args),
                   "form": "chosen: FP32-inner/" + ("double-word" if dw_used else "FP64") + "-refine, "
                           + algorithm_of(w, args),
                   "l2": "flushed (512 MB write) before every timed step", "replicas": world},
        "stencil_gbs": roofline["achieved"],
        "schwarz_iterations_per_step": statistics.mean(iters),
        "krylov_iterations_per_step": kry / args.steps,
        "nl_iterations_per_step": sum(s["nl_iterations"] for s in stats_p) / args.steps,
        "gmres_iterations_per_step": sum(s["gmres_iterations"] for s in stats_p) / args.steps,
        "ms_per_step_profiled": sum(ms_p) / args.steps,
        "strip_solve_phase_share": dict(zip(["residual", "krylov_pass1", "krylov_pass2", "epilogue", "waits"],
                                            [c / max(1.0, sum(prof["phase_cycles"])) for c in prof["phase_cycles"]])),
        "time_split_ms_per_step": {"strip_solve": prof["strip_solve_ms"] / args.steps,
                                   "interface": prof["interface_ms"] / args.steps,
                                   "other": prof["other_ms"] / args.steps},
        "plain_fp64": fp64,
        "speedup_vs_plain_fp64": (value / world) / fp64["value"] if fp64 else None,
        "rel_l2_chosen_vs_fp64": err,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": world * args.steps / (sum(e2e_ms) * 1e-3), "unit": "steps/s",
                "h2d_bytes_per_step": node_bytes, "d2h_bytes_per_step": node_bytes},
        "gpu_launches": prof["kernel_launches"],
        "clocks": clk,
    }
    if dist is not None:
        dist.destroy_process_group()
    return line


def extra_configs(args, local_rank):
    """The other single-GPU configurations, run after the headline one: the GPE trap with S_pade
    (gpe_trap) and the batched GPE instances (gpe_batch), with fewer steps, each with its own
    roofline, oracle sample, e2e and clocks; and the learned interface guess at its full size
    (learned_guess: 2000 training steps, 500 held-out steps)."""
    out = {}
    common = ["--warmup", "3", "--no-fp64", "--cpu-budget", str(args.cpu_budget), "--tol", str(args.tol)]
    if args.no_cpu:
        common.append("--no-cpu")
    runs = {"gpe_trap": run_ours, "gpe_batch": run_batch, "learned_guess": run_learned}
    for name, steps in (("gpe_trap", max(2, min(args.steps, 5))), ("gpe_batch", max(2, min(args.steps, 3))),
                        ("learned_guess", 1)):
        a = parse(["--workload", name, "--steps", str(steps)] + common)
        try:
            out[name] = runs[name](a, 0, 1, local_rank)
        except Exception as e:          # a failed extra line must not cost the headline line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_batch(args, rank, world, local_rank):
    """Batched GPE instances (gpe_batch): every instance stepped together, one persistent launch
    of the strip solver per Schwarz iteration over the strips of all unconverged instances."""
    import torch

    from paper_1603_05110_gb300 import binding, build, workloads as wl
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ws = wl.gpe_batch(args.instances)
    chosen = args.batch_form == "chosen"
    prms = []
    for w in ws:
        # chosen: preconditioned Schwarz (modal P^-1 per instance) with the double-word residual;
        # classical: the plain algorithm with the FP64 residual
        d = solver_params(w, args, binding.FP32_DW if chosen else binding.FP32_INNER)
        d.update(p=w.p, algorithm=binding.PRECONDITIONED if chosen else binding.CLASSICAL, tol=args.tol,
                 max_schwarz=args.max_schwarz, nl_tol=1e-11 if chosen else 1e-13, omega_rot=w.extra["omega"])
        prms.append(d)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    u0 = [torch.from_numpy(w.u0()).to(dev) for w in ws]
    V = [torch.from_numpy(w.V()).to(dev) for w in ws]
    b = binding.Batch(prms, u0, V, stream=stream)
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        b.step(1)
    warm_s = time.perf_counter() - t0

    def batch_steps(k):
        ms, stats = [], []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats.append(b.step(1))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, stats

    clocks = Clocks(local_rank)
    ms, stats = batch_steps(args.steps)          # the headline: the library's profiling off
    clk = clocks.stop()
    # the same number of steps again with profiling on: the strip solver's time for the roofline
    b.set_profiling(True)
    ms_p, stats_p = batch_steps(args.steps)
    prof = b.profile()
    b.set_profiling(False)
    bs, nblk = b.tuning()
    # e2e through the C-ABI with pinned host buffers: every instance's u_{n-1} in, step, every u_n out
    hu = [torch.empty(w.ny + 1, w.nx + 1, dtype=torch.complex128, pin_memory=True) for w in ws]
    for i in range(len(ws)):
        b.get_u(i, hu[i].numpy())
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for i in range(len(ws)):
            b.set_u(i, hu[i].numpy())
        b.step(1)
        for i in range(len(ws)):
            b.get_u(i, hu[i].numpy())
    e2e_s = time.perf_counter() - t0
    b.close()
    total_ms = sum(ms)
    nodes = sum(w.nodes() for w in ws)
    io_bytes = 16 * nodes
    # roofline: 68 B/node per strip-Krylov iteration of each instance's strips
    kb = 0.0
    for st in stats_p:
        for w, s1 in zip(ws, st):
            kb += KRYLOV_BYTES["fp32"] * (w.nx // w.n_strips + 1) * (w.ny + 1) * s1["krylov_iterations"]
    peaks, peak_kind = measured_peaks()
    t_strip = prof["strip_solve_ms"] * 1e-3
    roofline = {"kernel": "strip_solve_kernel<float> (batched)", "bound": "hbm", "achieved": kb / t_strip / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": kb / t_strip / 1e9 / peaks["hbm_gbs"],
                "peak_source": f"{peak_kind} hbm_gbs", "traffic": None,
                "share_of_step": prof["strip_solve_ms"] / sum(ms_p),
                "note": "68 B/node per strip-Krylov iteration x each instance's nodes per strip / strip-solver time"}
    its_mean = statistics.mean(statistics.mean(s2["last_schwarz_iterations"] for s2 in st) for st in stats)
    cpu = None
    if not args.no_cpu and world == 1:
        # bounded sample: the first 2 Schwarz iterations of step 1 of four instances (strip solves over
        # the host cores), scaled by each instance's Schwarz iterations per step measured here
        per_inst = []
        hi = host_info()
        for i in (0, 1, 2, 3):
            w = copy.deepcopy(ws[i])
            w.extra["relax"] = 0.6          # the oracle's plain fixed point diverges for the strongest beta
            a2 = parse(["--workload", "nls_well", "--tol", str(args.tol)])
            a2.p, a2.algorithm, a2.tc = w.p, "preconditioned" if chosen else "classical", "robin"
            r = oracle_steps(w, a2, 1, args.cpu_budget, max_iter_first=2)
            its_i = statistics.mean(st[i]["last_schwarz_iterations"] for st in stats)
            per_inst.append(r["steps"][0] / r["iterations"][0] * its_i)
        inst_s = statistics.mean(per_inst)
        cpu = {"value": 1.0 / inst_s, "unit": "instance-steps/s", "cores": r["processes"], "kind": "oracle",
               "sample": f"the first 2 Schwarz iterations of step 1 of instances 0-3 (strip solves over {r['processes']} "
                         f"worker processes), scaled by each instance's Schwarz iterations per step measured on the "
                         f"GPU ({statistics.mean(per_inst):.1f} s per instance-step); host {hi['cpu']}, {hi['nproc']} cores",
               "host": hi}
    line = {"metric": METRIC, "value": len(ws) * args.steps / (total_ms * 1e-3), "unit": "instance-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner Krylov + " + ("double-word f32x2" if chosen else "f64") + " residual, f64 interface",
            "data": "synthetic",
            "config": {"workload": f"gpe_batch: {len(ws)} GPE instances, meshes {min(w.nx for w in ws)}^2..{max(w.nx for w in ws)}^2 "
                                   f"cells, {sum(w.n_strips for w in ws)} strips, {nodes/1e6:.1f} M nodes, dt 0.002, "
                                   + ("preconditioned (modal P^-1 per instance)" if chosen else "classical")
                                   + f" Robin, tol {args.tol:g}",
                       "form": "chosen: FP32-inner/double-word-refine, preconditioned" if chosen
                               else "classical, FP32-inner/FP64-refine",
                       "l2": "flushed (512 MB write) before every timed step"},
            "autotuned": {"block_size": bs, "blocks_per_launch": nblk, "first_call_s": warm_s},
            "schwarz_iterations_per_step_max": max(max(s2["last_schwarz_iterations"] for s2 in st) for st in stats),
            "schwarz_iterations_per_step_mean": its_mean,
            "strip_solve_ms_per_step": prof["strip_solve_ms"] / args.steps,
            "strip_solve_launches_per_step": prof["strip_solve_launches"] / args.steps,
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": len(ws) * e2e_steps / e2e_s, "unit": "instance-steps/s", "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes},
            "gpu_launches": prof["kernel_launches"], "clocks": clk}
    return line


def learned_workload(args, beta, seed):
    """The GPE trap of the gpe_trap configuration at learn_n^2 cells and learn_strips strips
    (S_pade m = 8, Omega_rot 0.4, preconditioned), with the given beta."""
    from paper_1603_05110_gb300 import workloads as wl
    n, dt = args.learn_n, 0.001
    return wl.Workload("learned_gpe", -16.0, 16.0, -16.0, 16.0, n, n, args.learn_strips, dt, 1, lap=0.5,
                       kappa=-beta, p=2.0 * float(np.sqrt(1.0 / dt)), algorithm="preconditioned", potential="trap",
                       datum="ground_noise", seed=seed, extra={"tc": "pade", "pade_m": 8, "omega": 0.4})


def run_learned(args, rank, world, local_rank):
    """Learned interface guess (dd_cnn_*) on the GPE trap at 1024^2 cells with 32 strips: the plain
    solver generates training trajectories at seeded beta in [200, 800] (learn_train steps over
    learn_traj trajectories), the CNN is trained on the device to predict each step's converged
    interface vector from the previous three (a correction to the previous vector, the paper's
    guess), and a held-out trajectory at its own beta is solved step by step from the same state
    with four guesses: zero, the previous vector, linear extrapolation and the network's.  Schwarz
    iterations and time per step are reported for each; the learned time includes inference."""
    import torch

    from paper_1603_05110_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rng = np.random.default_rng(1603)
    betas = [float(b) for b in rng.uniform(200.0, 800.0, args.learn_traj + 1)]
    args.tc, args.pade_m = "pade", 8
    stream = torch.cuda.Stream(device=dev)

    def params_of(w):
        prm = solver_params(w, args, binding.FP32_DW if args.residual == "dw" else binding.FP32_INNER)
        prm["omega_rot"] = w.extra["omega"]
        return prm

    def trajectory(w, steps, keep_states=True):
        """States after steps 0..steps (keep_states) and the converged interface vectors of steps
        1..steps."""
        ntr = 2 * (w.n_strips - 1)
        us, gs = [torch.from_numpy(w.u0()).to(dev)], []
        its = []
        with binding.Solver(params_of(w), us[0], torch.from_numpy(w.V()).to(dev), stream=stream) as s:
            for _ in range(steps):
                out = torch.empty_like(us[0])
                its.append(s.step(1, out)["last_schwarz_iterations"])
                g = torch.empty(ntr, w.ny + 1, dtype=torch.complex128, device=dev)
                s.get_state(None, g)
                if keep_states:
                    us.append(out)
                gs.append(g)
        return us, gs, its

    # ---- training data: learn_traj trajectories, one beta each
    t0 = time.perf_counter()
    per = max(4, args.learn_train // args.learn_traj)
    train = []                                   # (g_{k-1}, g_{k-2}, g_{k-3}, g_k)
    gen_its = []
    for t in range(args.learn_traj):
        w = learned_workload(args, betas[t], 1603 + t)
        _, gs, its = trajectory(w, per, keep_states=False)
        gen_its += its
        train += [(gs[k - 1], gs[k - 2], gs[k - 3], gs[k]) for k in range(3, len(gs))]
    gen_s = time.perf_counter() - t0
    # ---- held-out trajectory (its own beta); its states are the starting points of the solves
    w = learned_workload(args, betas[-1], 1603 + args.learn_traj)
    t0 = time.perf_counter()
    us, gs, _ = trajectory(w, args.learn_eval + 4)
    gen_s += time.perf_counter() - t0
    ntr = 2 * (w.n_strips - 1)
    # ---- training on the device (Adam), shuffled samples, learning rate halved each epoch
    net = binding.CNN(ntr, w.ny + 1, stream=stream, base=binding.CNN.BASE_PREVIOUS)
    net.set_params(binding.CNN.init_params(seed=7, last_scale=0.1))
    t0 = time.perf_counter()
    losses = []
    order_rng = np.random.default_rng(7)
    for ep in range(args.learn_epochs):
        lr = 1e-3 * 0.5 ** ep
        for i in order_rng.permutation(len(train)):
            losses.append(net.train_step(*train[i], lr=lr))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del train

    # ---- held-out steps: each solved from the same state with each guess
    kinds = ("zero", "previous", "extrapolated", "learned")
    res = {k: [] for k in kinds}
    g0 = torch.empty(ntr, w.ny + 1, dtype=torch.complex128, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = Clocks(local_rank)
    with binding.Solver(params_of(w), us[0], torch.from_numpy(w.V()).to(dev), stream=stream) as s:
        for k in range(3, 3 + args.learn_eval):
            # state after step k + 1 (us[k + 1]); the step to solve is k + 2, whose vector is gs[k + 1]
            for kind in kinds:
                s.set_state(us[k + 1], gs[k], k + 1)
                with torch.cuda.stream(stream):
                    flush.zero_()           # every solve starts from a cold L2
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if kind == "learned":
                    net.guess(gs[k], gs[k - 1], gs[k - 2], g0)
                    st = s.solve_interface(g0)
                elif kind == "extrapolated":
                    with torch.cuda.stream(stream):     # the solver reads g0 on this stream
                        g0.copy_(2 * gs[k] - gs[k - 1])
                    st = s.solve_interface(g0)
                elif kind == "zero":
                    with torch.cuda.stream(stream):
                        g0.zero_()
                    st = s.solve_interface(g0)
                else:
                    st = s.solve_interface(gs[k])
                e1.record(stream)
                e1.synchronize()
                res[kind].append((st["last_schwarz_iterations"], e0.elapsed_time(e1)))
    clk = clocks.stop()
    net.close()
    if rank != 0:
        return None
    its = {k: statistics.mean(v[0] for v in res[k]) for k in res}
    ms = {k: statistics.mean(v[1] for v in res[k]) for k in res}
    nl = len(losses)
    line = {"metric": METRIC, "value": 1e3 / ms["learned"], "unit": "steps/s", "n_gpus": world,
            "steps": len(res["learned"]), "warmup": 0, "ms_per_step": ms["learned"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 inner Krylov + " + ("double-word f32x2" if args.residual == "dw" else "f64")
                     + " residual, f64 interface; CNN bf16 operands / f32 accumulate", "data": "synthetic",
            "config": {"workload": f"learned_guess: GPE trap, {w.nx}x{w.ny} cells on (-16,16)^2, {w.n_strips} strips, "
                                   f"preconditioned Schwarz, S_pade m=8, Omega_rot 0.4, dt={w.dt}, interface tol {args.tol:g}; "
                                   f"training: {args.learn_traj} trajectories x {per} steps at beta "
                                   + ", ".join(f"{b:.0f}" for b in betas[:-1])
                                   + f"; held out: {len(res['learned'])} steps at beta {betas[-1]:.0f}",
                       "note": "each held-out step solved from the same state with each guess; L2 flushed "
                               "(512 MB write) before every timed solve; the network predicts a correction to "
                               "the previous step's vector"},
            "schwarz_iterations_per_step": {f"{k}_guess": its[k] for k in kinds},
            "ms_per_step_by_guess": {f"{k}_guess": ms[k] for k in kinds},
            "learned_vs_previous_speedup": ms["previous"] / ms["learned"],
            "learned_vs_zero_speedup": ms["zero"] / ms["learned"],
            "training": {"updates": nl, "epochs": args.learn_epochs, "samples": nl // max(1, args.learn_epochs),
                         "loss_first_100": statistics.mean(losses[:100]) if losses else None,
                         "loss_last_100": statistics.mean(losses[-100:]) if losses else None, "seconds": train_s},
            "generation_s": gen_s, "generation_schwarz_iterations_mean": statistics.mean(gen_its),
            "clocks": clk}
    return line


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.workload == "gpe_batch":
        line = run_batch(args, rank, world, local_rank)
        if line is not None and rank == 0:
            print(json.dumps(line), flush=True)
    elif args.workload == "learned_guess":
        line = run_learned(args, rank, world, local_rank)
        if line is not None:
            print(json.dumps(line), flush=True)
    else:
        line = run_ours(args, rank, world, local_rank)
        if line is not None:
            if world == 1 and args.workload == "nls_well" and not args.no_extra:
                line["configs"] = extra_configs(args, local_rank)
            print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()

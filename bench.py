"""Benchmark of the space-time PDHG iteration (Algorithm 1) on GB300.

One "step" is one PDHG iteration over the whole space-time grid of the
workload: primal step, residual, preconditioned dual step and extrapolation
for every (dof, time slice) at once.  The metric is space-time
cell-iterations per second (dofs x equation slices x iterations / s).

Default workload (N = 1): 2D Burgers u_t + (u^2/2)_x + (u^2/2)_y = 0 on a
periodic 1024 x 1024 grid, 256 time slices (268,435,456 space-time cells),
h_t = h_x (T = pi/2), backward Euler + global Lax-Friedrichs, float32 fields,
u0 = 8 seeded random Fourier modes.  The state (u, phi, phit, spectrum: about 4.3 GB) is far larger
than L2, so consecutive iterations stream it from HBM.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 runs under torch.distributed.run: every rank solves its own replica of
the workload (the method has no data-parallel split across GPUs here;
"replicas only"), the timed region is bracketed by barriers and the slowest
rank's time is used.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pdhg_workloads as W  # noqa: E402

METRIC = "PDHG space-time cell-iters/s & HBM %peak; time-to-residual 1e-6 vs plain GPU"
UNIT = "cell-iters/s"


def workload(name: str):
    if name == "burgers2d":
        return W.burgers_2d(n=1024, nt=256, tau=(0.15, 0.1, 0.15, 0.99))
    if name == "burgers2d_small":
        return W.burgers_2d(n=256, nt=64, tau=(0.15, 0.1, 0.15, 0.99))
    if name == "burgers2d_nt32":                      # profiling case: 134 MB per field (> L2)
        return W.burgers_2d(n=1024, nt=32, tau=(0.15, 0.1, 0.15, 0.99))
    if name == "burgers2d_nt64":                      # profiling case with the full run's t-chunking
        return W.burgers_2d(n=1024, nt=64, tau=(0.15, 0.1, 0.15, 0.99))
    if name == "dg_p2":
        return W.burgers_dg_p2(tau=(0.2, 0.1, 0.2, 0.99)).replace(c=0.5)
    if name == "advection":
        return W.advection_upwind_be(tau=(1.4, 0.1, 0.35, 0.99))
    if name == "heat":                                # Table 1's finest mesh, Sec. 4.1
        return W.heat_table1(1024, 256)
    if name == "transport2d":                         # 2D linear transport: the fused path converges
        return W.burgers_2d(n=1024, nt=64).replace(name="transport2d_1024x1024x64", alpha=0.0, beta=1.0,
                                                    space="fd_upwind", lf_a=1.0, c=1.0, tau_u=0.5,
                                                    tau_phi=0.5, tau_u0=0.1)
    raise ValueError(name)


# ---------------------------------------------------------------------------
# distributed helpers (replicas only: no data-path collective)
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(local_units: float, local_ms: float, group=None):
    """Whole-job throughput: units summed over ranks / the slowest rank's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local_units / (local_ms * 1e-3), local_ms
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        self.gpu = gpu_index
        self.path = path
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [ln for ln in out.splitlines() if ln.strip()]
        if self.path:
            with open(self.path, "w") as f:
                f.write(self.FIELDS + "\n" + "\n".join(self.lines) + "\n")

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            t = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(t[1]))
                smax = float(t[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, t[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


# ---------------------------------------------------------------------------
# roofline bookkeeping: algorithmic bytes per launch of each stage
# ---------------------------------------------------------------------------

def stage_bytes(p, esz: int):
    """Compulsory HBM bytes of one launch of each stage: every input read once,
    every output written once (sizes from the array shapes)."""
    S, nt = p.ndof, p.nt
    lines = 3 if p.space == "dg_p2_lf" else (p.ny if p.dims == 2 else 1)
    spec = nt * lines * (p.nx // 2 + 1) * 2 * esz          # complex spectrum, all slices
    u = (nt + 1) * S * esz
    f = nt * S * esz
    lam = S * esz
    return {
        "primal": u + f + u + 3 * lam + 2 * lam,            # read u, phit; write u; lambda row
        "residual_fft": u + spec,                           # read u; write spectrum
        "fft_y": 2 * spec,                                  # read + write spectrum
        "tsolve": 4 * spec,                                 # forward sweep r/w, backward r/w
        "dual": spec + f + 2 * f,                           # read spectrum, phi; write phi, phit
        "fused_rows": u + spec,                             # rows-R: read u; write X
        "fused_cols": spec + spec + 2 * spec,               # read X, write Zx, spill w/r
    }


# Algorithmic bytes of one pass of the whole path per cell-iteration, by element size:
# u and phit read, u written (12 B in float32), the t-solve's one spill round trip
# (8 B), phi read and phi, phit written (12 B).
ALG_BYTES_PER_CELL = {4: 32, 8: 64}

KERNEL_SOURCES = {"primal": "kernels_plain.cu", "residual_fft": "kernels_plain.cu",
                  "fft_y": "kernels_plain.cu", "tsolve": "kernels_plain.cu",
                  "dual": "kernels_plain.cu", "fused_rows": "kernels_fused2d.cu",
                  "fused_cols": "kernels_fused2d.cu"}
# the fused 2D path runs its own primal and dual kernels
FUSED_SOURCES = dict(KERNEL_SOURCES, primal="kernels_fused2d.cu", dual="kernels_fused2d.cu")


def traffic_for(stage: str, workload_name: str, fused: bool = False):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        db = json.load(open(path))
        ent = db.get(workload_name, {}).get(stage)
        if not ent:
            return None
        src = os.path.join(ROOT, "paper_2207_07234_gb300", "csrc", (FUSED_SOURCES if fused else KERNEL_SOURCES)[stage])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if ent.get("src_sha") != sha:
            return None
        return ent["dram_bytes_per_launch"]
    except Exception:
        return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(p, nt_sample=8):
    """The workload cut to its first nt_sample time slices (same grid, same u0)."""
    return p.replace(nt=nt_sample, T=p.ht * nt_sample)


CPU_SAMPLE_ITERS = 16          # about 10 s of single-core oracle work on the 8-slice sample


def time_oracle(p, iters=3, warm=1):
    from oracle import pdhg as opdhg
    q = oracle_sample(p)
    st = opdhg.initial_state(q)
    for _ in range(warm):
        opdhg.step(q, st)
    t0 = time.perf_counter()
    for _ in range(iters):
        opdhg.step(q, st)
    dt = time.perf_counter() - t0
    return q.cells_per_iter * iters / dt, q, dt


def _oracle_worker(args):
    """One host process: the oracle on the workload's 8-slice sample (single-threaded
    numpy), timed between two barriers shared by all processes."""
    name, iters, warm, bar = args
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    from oracle import pdhg as opdhg
    q = oracle_sample(workload(name))
    st = opdhg.initial_state(q)
    for _ in range(warm):
        opdhg.step(q, st)
    bar.wait()
    t0 = time.perf_counter()
    for _ in range(iters):
        opdhg.step(q, st)
    dt = time.perf_counter() - t0
    return q.cells_per_iter * iters, dt


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle_all_cores(name, iters, warm=1, procs=None):
    """The oracle on every host core at once: one spawned process per core, each on its
    own copy of the 8-slice sample; throughput = all processes' cell-iterations / the
    slowest process's time.  Returns (value, processes, seconds)."""
    import multiprocessing as mp
    n = procs or host_cores()
    ctx = mp.get_context("spawn")             # no fork after CUDA initialisation
    with ctx.Manager() as m:
        bar = m.Barrier(n)
        with ctx.Pool(n) as pool:
            res = pool.map(_oracle_worker, [(name, iters, warm, bar)] * n)
    cells = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return cells / dt, n, dt


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args):
    """The oracle (float64 numpy, as it stands) on every host core: one process per
    core, each on the workload's 8-slice sample, `steps` timed iterations after
    `warmup` untimed ones."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    p = workload(args.workload)
    q = oracle_sample(p)
    value, n, dt = time_oracle_all_cores(args.workload, args.steps, warm=args.warmup)
    sample = (f"{q.name.replace(str(p.nt), str(q.nt))}: the workload cut to its first {q.nt} "
              f"time slices, {args.steps} oracle iterations in each of {n} processes (one per host core)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": p.name, "oracle_sample_slices": q.nt},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def optional_leg(name, fn):
    """Runs one of the legs that follow the timed iterations; an exception there is
    recorded in the result line (and on stderr) instead of costing the line itself."""
    try:
        return fn()
    except Exception as err:                      # noqa: BLE001 - any failure of the leg
        print(f"bench: the {name} leg failed: {type(err).__name__}: {err}", file=sys.stderr)
        return {"error": f"{type(err).__name__}: {err}"}


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2207_07234_gb300 import binding

    p = workload(args.workload)
    esz = 4 if args.precision == "fp32" else 8
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    solver = binding.Solver(p, precision=args.precision, path=args.path, device=dev, stream=stream)
    path = solver.info()["path"]

    # warm-up
    solver.iterate(args.warmup)
    torch.cuda.synchronize()
    solver.launches(reset=True)
    solver.set_profiling(True)
    solver.stage_times()                      # clear

    barrier()
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk_path = args.clock_log
    with ClockSampler(gpu_index(local), clk_path) as clk:
        start.record(stream)
        solver.iterate(args.steps)
        end.record(stream)
        torch.cuda.synchronize()
    barrier()
    local_ms = start.elapsed_time(end)
    launches = solver.launches(reset=True)
    stages = solver.stage_times()
    solver.set_profiling(False)
    units = p.cells_per_iter * args.steps
    value, max_ms = aggregate(units, local_ms)

    # roofline: the whole iteration against the algorithmic bytes of one pass of the
    # path (32 B per cell-iteration in float32, 64 B in float64: u and phit read and u
    # written, one spill round trip of the t-solve, phi read and phi, phit written),
    # timed as ms_per_step; then every stage against its own compulsory bytes
    sb = stage_bytes(p, esz)
    dom = max(stages, key=lambda k: stages[k][0]) if stages else None
    peak, peak_kind = measured_peaks()
    roof = None
    if dom:
        step_bytes = ALG_BYTES_PER_CELL[esz] * p.cells_per_iter
        step_s = local_ms / args.steps * 1e-3
        achieved = step_bytes / step_s / 1e9
        per = {}
        traffic_sum, traffic_ok = 0.0, True
        for k, (ms, n) in stages.items():
            tr = traffic_for(k, p.name, path == "fused")
            per[k] = {"algorithmic_bytes_per_launch": sb.get(k), "avg_launch_ms": ms / n,
                      "launches_per_step": n / args.steps,
                      "achieved_gbs": (sb[k] / (ms / n * 1e-3) / 1e9) if k in sb else None,
                      "frac": (sb[k] / (ms / n * 1e-3) / 1e9 / peak) if k in sb else None,
                      "traffic": tr, "ms_share": round(ms / sum(x[0] for x in stages.values()), 4)}
            if tr is None:
                traffic_ok = False
            else:
                traffic_sum += tr * n / args.steps
        per_dom = per[dom]
        roof = {"bound": "hbm", "kernel": "iteration (all kernels of one step)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_sum if traffic_ok else None,
                "algorithmic_bytes_per_cell": ALG_BYTES_PER_CELL[esz],
                "algorithmic_bytes_per_step": step_bytes,
                "measured_dram_bytes_per_cell": (traffic_sum / p.cells_per_iter) if traffic_ok else None,
                "measured_dram_frac": (traffic_sum / step_s / 1e9 / peak) if traffic_ok else None,
                "peak_source": peak_kind,
                "dominant_kernel": dict(per_dom, kernel=dom),
                "stages": per}
    solver.close()
    del solver
    torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: upload u0 from pinned host
    # memory, K iterations with one residual read-back, terminal slice to pinned host
    e2e = None
    if not args.no_e2e:
        u0_host = torch.from_numpy(np.ascontiguousarray(p.u0, dtype=np.float64)).pin_memory()
        out_host = torch.empty(p.slice_shape, dtype=torch.float32 if esz == 4 else torch.float64).pin_memory()
        q = p.replace(u0=u0_host.numpy())
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = binding.Solver(q, precision=args.precision, path=args.path, device=dev, stream=stream)
        try:
            s2.iterate(args.steps, tol=0.0, check_every=args.steps)
        except binding.PdhgError as err:          # a diverging problem still counts its work
            if err.status not in (-4, -5):
                raise
        s2.get_host("u_terminal", out=out_host.numpy())
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        barrier()
        s2.close()
        e2e_val, _ = aggregate(units, e2e_s * 1e3)
        h2d = p.ndof * 8 + (p.nx if p.gamma_half is not None else 0) * 8
        d2h = p.ndof * esz + 6 * 8
        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps}

    def cpu_leg():
        v1, q, dt1 = time_oracle(p, iters=CPU_SAMPLE_ITERS)
        va, n, dta = time_oracle_all_cores(args.workload, CPU_SAMPLE_ITERS // 2)
        return {"value": va, "unit": UNIT, "cores": n, "kind": "oracle",
                "sample": f"{p.name} cut to its first {q.nt} time slices: {CPU_SAMPLE_ITERS // 2} oracle "
                          f"iterations in each of {n} processes, one per host core ({dta:.1f} s)",
                "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                                "sample": f"{CPU_SAMPLE_ITERS} oracle iterations in one process ({dt1:.1f} s)"}}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = optional_leg("cpu_baseline", cpu_leg)

    ttr = None
    if args.ttr and rank == 0:
        ttr = [optional_leg(f"time_to_residual {w}",
                            lambda w=w: time_to_residual(binding, workload(w), device=dev, stream=stream))
               for w in args.ttr.split(",") if w]

    batch = None
    if not args.no_batch and rank == 0:
        batch = optional_leg("batch", lambda: batch_leg(binding, device=dev, stream=stream))

    nonlin = None
    if not args.no_nonlinear and rank == 0 and args.workload == "burgers2d" and args.precision == "fp32":
        nonlin = optional_leg("nonlinear", lambda: nonlinear_leg(binding, device=dev, stream=stream))

    grad = None
    if not args.no_gradient and rank == 0:
        grad = optional_leg("gradient", lambda: gradient_leg(binding, device=dev, stream=stream))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if esz == 4 else "f64",
                "data": "synthetic",
                "config": {"workload": p.name, "nx": p.nx, "ny": p.ny, "nt": p.nt,
                           "cells_per_iter": p.cells_per_iter, "scheme": f"{p.time}+{p.space}",
                           "path": path, "l2": "state larger than L2 (no flush needed)",
                           "parallelism": f"replicas{ws}"},
                "gpu_launches": launches, "launches_per_iter": launches / args.steps,
                "clocks": clk.summary(), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e}
        if ttr:
            line["time_to_residual"] = ttr
        if batch:
            line["batch"] = batch
        if nonlin:
            line["nonlinear"] = nonlin
        if grad:
            line["gradient"] = grad
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batch_leg(binding, steps=10, warmup=3, device=None, stream=None):
    """The 256-instance batch of mixed 1D problems (pdhg_workloads.batch_instances,
    float32): cell-iterations per second of the shared launches over all instances
    (fixed iteration count, no residual checks), with the algorithmic HBM rate of
    the whole iteration (sum over instances of the plain path's stage bytes)."""
    import torch
    probs = W.batch_instances()
    cells = sum(p.cells_per_iter for p in probs)
    nbytes = 0
    for p in probs:
        b = stage_bytes(p, 4)
        nbytes += b["primal"] + b["residual_fft"] + b["tsolve"] + b["dual"]
    s = stream if stream is not None else torch.cuda.current_stream()
    with binding.Batch(probs, precision="fp32", device=device, stream=s) as bt:
        bt.iterate(warmup)
        bt.launches(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        bt.iterate(steps)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        launches = bt.launches() / steps
    # CUDA-graph replay against launch by launch, with a residual check every `steps`
    # iterations (instances whose residual stops being finite leave at a check, so both
    # runs take the same fresh batch through the same sequence: an untimed chunk, which
    # also captures the graph, then a timed one)
    graph = {"check_every": steps}
    for use_graph in (False, True):
        with binding.Batch(probs, precision="fp32", device=device, stream=s) as bt:
            bt.set_graphs(use_graph)
            bt.iterate(steps, tol=0.0, check_every=steps)
            _, st = bt.iterate(0)
            torch.cuda.synchronize()
            e0.record(s)
            bt.iterate(steps, tol=0.0, check_every=steps)
            e1.record(s)
            torch.cuda.synchronize()
            graph["graph_ms_per_iter" if use_graph else "launch_by_launch_ms_per_iter"] = e0.elapsed_time(e1) / steps
            graph["active_instances"] = int(np.sum(np.asarray(st) == 0))
    peak, src = measured_peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"workload": f"{len(probs)} mixed 1D instances, seed 20723", "instances": len(probs),
            "cells_per_iter": cells, "steps": steps, "ms_per_iter": ms, "value": cells / (ms * 1e-3),
            "unit": UNIT, "launches_per_iter": launches, "algorithmic_bytes_per_iter": nbytes,
            "achieved_gbs": gbs, "frac": gbs / peak, "peak_source": src,
            "graph": graph}


def gradient_leg(binding, iters=200, device=None, stream=None):
    """Cost per iteration of the forward and the adjoint solve of the gradient at the
    gradient workload's own shape: viscous Burgers 2048 x 1024, BDF2, nu = 1e-3, float32,
    plain path.  Algorithm 1 does not converge on that configuration, so fixed iteration
    counts are timed (small steps tau = 0.05 keep the iterates finite over them; the cost
    of an iteration does not depend on the steps): the forward iterations alone (device
    time by CUDA events), then pdhg_solve_gradient with (n, n) and (2n, 2n)
    forward/adjoint iterations, whose difference in wall-clock time is n forward plus n
    adjoint iterations."""
    import torch
    p = W.viscous_burgers().replace(tau_u=0.05, tau_phi=0.05, tau_u0=0.05)
    s = stream if stream is not None else torch.cuda.current_stream()
    out = {"workload": p.name + f"_bdf2_nu{p.nu:g}", "cells_per_iter": p.cells_per_iter, "precision": "fp32",
           "iterations": iters}
    try:
        with binding.Solver(p, precision="fp32", path="plain", device=device, stream=s) as sv:
            # device time per iteration: iters iterations plus one residual check replayed
            # as one CUDA graph (the first call captures it), timed by events on the stream
            sv.iterate(iters, tol=0.0, check_every=iters)
            torch.cuda.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            sv.iterate(iters, tol=0.0, check_every=iters)
            e.record(s)
            torch.cuda.synchronize()
            fwd = a.elapsed_time(e) * 1e-3 / iters
        target = np.zeros(p.slice_shape)
        tg = []
        for n in (iters, 2 * iters):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            binding.solve_gradient(p, target, tol=0.0, max_iters=n, adj_tol=0.0, adj_max_iters=n, check_every=n,
                                   precision="fp32", device=device, stream=s)
            torch.cuda.synchronize()
            tg.append(time.perf_counter() - t0)
        both = (tg[1] - tg[0]) / iters
        adj = both - fwd
        out.update({"forward_ms_per_iter": fwd * 1e3, "adjoint_ms_per_iter": adj * 1e3,
                    "forward_value": p.cells_per_iter / fwd, "adjoint_value": p.cells_per_iter / adj,
                    "unit": UNIT, "gradient_call_seconds": tg})
    except binding.PdhgError as err:
        out["status"] = f"stopped: {err}"
    out["converged"] = gradient_converged(binding, device=device, stream=s)
    return out


def gradient_converged(binding, device=None, stream=None):
    """The gradient workload's shape and scheme before the shock (T = 0.5 instead of 2),
    with the exact time operator (PDHG_FLAG_EXACT_TIME_PRECOND; with T_t the admissible
    BDF2 steps shrink as nt^{-1/2} and Algorithm 1 makes no progress here): forward solve to
    relative Res 1e-6 in float64 and by the mixed solve, and the float32 gradient of
    |u^nt - target|^2, target = 0.5 + 0.9 sin(x - 1): forward to float32's floor (at most
    4000 iterations), adjoint 30,000 iterations (its multipliers converge more slowly than
    the forward state; at 30,000 the float32 gradient agrees with a float64 one to 1e-5)."""
    import torch
    p = W.viscous_burgers(T=0.5).replace(tprec="exact", tau_u=0.45, tau_phi=0.45, tau_u0=0.45)
    out = {"workload": p.name + f"_bdf2_nu{p.nu:g}_T{p.T:g}_exact_time_operator", "tol": 1e-6}
    try:
        with binding.Solver(p, precision="fp64", path="plain", device=device, stream=stream) as s:
            r0 = float(s.residual()[0])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n = s.iterate(20000, tol=1e-6, check_every=100, relative=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            r = s.residual()
            out["forward_fp64"] = {"seconds": dt, "iterations": int(n), "rel_res": max(r[0], r[1]) / r0}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sm, its = binding.solve_mixed(p, tol=1e-6, relative=True, check_every=100, max_iters=20000, device=device,
                                      stream=stream)
        torch.cuda.synchronize()
        out["forward_mixed"] = {"seconds": time.perf_counter() - t0, "iterations": [int(v) for v in its]}
        sm.close()
        target = 0.5 + 0.9 * np.sin(W.fd_nodes(p.nx, p.lx) - 1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss, du0, dnu, its = binding.solve_gradient(p, target, tol=1e-7, max_iters=4000, adj_tol=0.0,
                                                     adj_max_iters=30000, check_every=100, precision="fp32",
                                                     device=device, stream=stream)
        torch.cuda.synchronize()
        out["gradient_fp32"] = {"seconds": time.perf_counter() - t0, "iterations": [int(v) for v in its],
                                "loss": loss, "dloss_dnu": dnu, "dloss_du0_norm": float(np.linalg.norm(du0))}
    except binding.PdhgError as err:
        out["status"] = f"stopped: {err}"
    return out


def nonlinear_leg(binding, tol=1e-6, device=None, stream=None, alg1_iters=1000):
    """The benchmark workload itself (2D Burgers 1024^2 x 256, BE + global LF, shocks form
    inside the horizon) to relative Res <= tol.  Algorithm 1 from [u0, 0, 0] does not
    converge on it (its relative residual over a fixed budget of float32 fused iterations
    is reported); Algorithm 3 (Sec. 3.5: one time step at a time, each step's u^0 pinned
    to the previous step's value) does.  Each step runs to tol * ||A(u_init)|| / sqrt(T),
    so that the assembled space-time solution has relative Res <= tol; that Res is then
    evaluated on the whole space-time problem (float64 residual norms).  Legs: Algorithm 3
    in float64 on the plain path (the plain-GPU comparator), in float32 (each step to
    its tolerance or float32's rounding floor) and mixed (each step in float32 to its
    floor, then float64 to the tolerance)."""
    import torch
    p = workload("burgers2d")
    out = {"workload": p.name, "tol": tol, "relative_to": "||A(u_init)||"}
    with binding.Solver(p, precision="fp64", path="plain", device=device, stream=stream) as s:
        r0 = float(s.residual()[0])
    hist, status = [], "max_iters"
    s = binding.Solver(p, precision="fp32", path="auto", device=device, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        for _ in range(alg1_iters // 100):
            s.iterate(100, tol=0.0, check_every=100)
            r = s.residual()
            hist.append(max(float(r[0]), float(r[1])) / r0)
    except binding.PdhgError as err:
        status = f"stopped: {binding.STATUS.get(err.status)}"
    torch.cuda.synchronize()
    out["alg1_fp32"] = {"seconds": time.perf_counter() - t0, "iterations": 100 * len(hist), "status": status,
                        "path": s.info()["path"], "rel_res_every_100": hist}
    s.close()
    del s
    torch.cuda.empty_cache()
    q = p.replace(init="pinned", tau_u=0.55, tau_u0=0.55, tau_phi=0.55)
    # a step's Res is the norm at one time (weight w_x, no h_t; Sec. 3.5), so the assembled
    # Res^2 = h_t * sum of the steps' Res^2 <= T max step Res^2: steps to tol * r0 / sqrt(T)
    # give a relative Res <= tol.  float32 steps cannot reach that (float32's rounding
    # floor, reached in about 60 iterations): they are capped at 200 iterations, about what
    # float64 steps need
    tol_step = tol * r0 / float(np.sqrt(p.T))
    sols = {}
    for label, prec, chk, cap in (("alg3_fp32", "fp32", 20, 200), ("alg3_mixed", "mixed", 10, 4000),
                                  ("alg3_fp64_plain", "fp64", 10, 4000)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, per = binding.solve_one_step(q, tol=tol_step, max_iters_per_step=cap, check_every=chk, precision=prec,
                                        device=device, stream=stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        with binding.Solver(p, precision="fp64", path="plain", device=device, stream=stream) as s:
            s.set("u", u.to(torch.float64))
            r = s.residual()
        rel = float(r[0]) / r0
        out[label] = {"seconds": dt, "iterations": int(sum(per)), "max_per_step": int(max(per)),
                      "status": "converged" if rel <= tol else "floor", "rel_res": rel,
                      "path": {"fp32": "fused float32 steps (one time step at a time)",
                               "mixed": "one time step at a time, each step float32 on the fused path to its "
                                        "floor, then float64 on the plain path",
                               "fp64": "plain (one time step at a time)"}[prec]}
        sols[label] = u
    # the float32 and mixed solutions against the float64 one (relative L-inf over all slices)
    ref = sols["alg3_fp64_plain"].to(torch.float64)
    scale = float(ref.abs().max())
    for label in ("alg3_fp32", "alg3_mixed"):
        out[label]["u_rel_linf_vs_fp64"] = float((sols[label].to(torch.float64) - ref).abs().max()) / scale
    del sols, ref
    torch.cuda.empty_cache()
    return out


def time_to_residual(binding, p, tol=1e-6, check_every=50, max_iters=20000, device=None, stream=None):
    """Wall time and iterations to relative Res <= tol for the float32 default path, the
    same with the t-solve recurrence in float64 (fp32_t64: whether float32's floor comes
    from that recurrence), and the plain float64 GPU path (the comparator named by the
    metric).  Iterates in chunks
    of 20 checks; a residual that has not dropped by 5% over three chunks is reported as
    the precision's floor instead of running to max_iters.  A third leg times the
    mixed-precision solve (float32, then float64 from the widened state)."""
    import torch
    out = {"workload": p.name, "tol": tol, "relative_to": "||A(u_init)||", "check_every": check_every}
    chunk = 20 * check_every
    legs = [("fp32", "fp32", "auto", False), ("fp32_t64", "fp32", "auto", True), ("fp64_plain", "fp64", "plain", False)]
    for label, prec, path, t64 in legs:
        try:
            s = binding.Solver(p, precision=prec, path=path, device=device, stream=stream, t64=t64)
        except binding.PdhgError as err:            # e.g. a t-recurrence variant the scheme does not take
            out[label] = {"status": f"unsupported: {err}"}
            continue
        r0 = float(s.residual()[0])
        scale0 = r0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        status, it, hist = "max_iters", 0, []
        try:
            while it < max_iters:
                done = s.iterate(min(chunk, max_iters - it), tol=tol, check_every=check_every, relative=True)
                it += done
                r = s.residual()
                hist.append(max(float(r[0]), float(r[1])) / r0)
                if r[0] <= tol * r0 and r[1] <= tol * r0:
                    status = "converged"
                    break
                if len(hist) >= 4 and hist[-1] > 0.95 * hist[-4]:
                    status = "floor"
                    break
        except binding.PdhgError as err:
            status = f"stopped: {binding.STATUS.get(err.status)}"
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        r = s.residual()
        out[label] = {"seconds": dt, "iterations": it, "status": status, "path": s.info()["path"],
                      "rel_res": [float(r[0]) / r0, float(r[1]) / r0]}
        s.close()
        del s
        torch.cuda.empty_cache()
    # float32 until the tolerance or its floor, then float64 (pdhg_solve_mixed); the
    # creation of both handles is inside the timed call
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    try:
        s, its = binding.solve_mixed(p, tol=tol, relative=True, check_every=check_every, max_iters=max_iters,
                                     device=device, stream=stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        r = s.residual()
        r0 = scale0
        status = "converged" if r[0] <= tol * r0 and r[1] <= tol * r0 else "max_iters"
        out["mixed"] = {"seconds": dt, "iterations": its, "status": status, "path": "float32 then float64 plain",
                        "rel_res": [float(r[0]) / r0, float(r[1]) / r0]}
        s.close()
    except binding.PdhgError as err:
        out["mixed"] = {"status": f"stopped: {binding.STATUS.get(err.status)}"}
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="burgers2d")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--path", default="auto", choices=["auto", "plain", "fused"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-instance batch leg")
    ap.add_argument("--no-gradient", action="store_true", help="skip the gradient-workload timing leg")
    ap.add_argument("--no-nonlinear", action="store_true",
                    help="skip the converged solve of the workload itself (Algorithm 3, float32 and float64)")
    ap.add_argument("--clock-log", default=None, help="also write the raw nvidia-smi clock samples to this CSV")
    ap.add_argument("--ttr", default="advection,heat,transport2d",
                    help="comma-separated workloads for the time-to-residual comparison ('' = skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

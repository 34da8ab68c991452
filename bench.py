"""Benchmark: interior point solves per second on the 1025^2 Poisson control sweep.

One step = one complete solve (Algorithm A.1 with preconditioned Krylov Newton
solves, every stage in libipm's CUDA kernels) of one cell of the sweep
alpha in {1e-2, 1e-4, 1e-6} x beta in {1e-2, 1e-3, 1e-4} (steps rotate over the
nine cells), Gaussian-sum y_d, u in [-30, 30], y <= 0.1, stopped at relative KKT
residual 1e-6. The headline value uses the mixed-precision path; the all-FP64
path is timed beside it on the same cells.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own share of the sweep (replicas,
no collective on the data path); value = all solves / max-over-ranks time.
The reference arm (--impl reference) is the oracle: plain FP64 CPU code run on this
host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IPM solves/s & p50/p99 latency, mixed vs FP64 GPU at 1e-6 rel. KKT residual"
N_DEFAULT = 1025

# Algorithmic bytes per unknown node per Krylov iteration of the whole mixed-precision
# solve (2D, FGMRES + P_T): each pass reads its operands and writes its result once --
# saddle operator 88 B (FP64), Chebyshev 20 steps x 5 values x 4 B + 24 B, z-block 48 B,
# coupling 40 B, six V-cycles of 47 values x 4 B x 4/3 (levels) plus the (M + Theta_y)
# product, and FGMRES orthogonalisation: about 2.3 KB.
SOLVE_BYTES_PER_NODE_ITER = 2300.0

# DRAM traffic per launch of the kernels the roofline may name (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture, the average over the launches of that kernel
# group), valid while the hashed source region of the kernels is unchanged. The middle-level
# tiles: the pre- and post-smoothing launches on the 513^2, 257^2 and 129^2 levels (captured
# in a 513^2 solve, whose tiled levels are exactly these and use the same tile shapes).
NCU_TRAFFIC = {
    "mid_level_tiles": {"bytes": (2116352 + 545792 + 152576 + 3456768 + 886272 + 242432) / 6.0,
                        "source": ("paper_1806_05896_gb300/csrc/k_mg_fused.cu",
                                   "// Register-blocked FP32 tile kernels",
                                   "// One CTA, all coarse levels in shared memory"),
                        "sha256": "00383ae4a950bfdd8fd27e2a90f8dd804e2c38663a5e0434477e27b72b020f46"},
}


def traffic_if_current(name):
    """The recorded DRAM bytes per launch of a kernel group, or None once its source changed."""
    import hashlib
    t = NCU_TRAFFIC.get(name)
    if not t:
        return None
    path, start, end = t["source"]
    with open(os.path.join(ROOT, path)) as f:
        src = f.read()
    i, j = src.find(start), src.find(end)
    if not 0 <= i < j or hashlib.sha256(src[i:j].encode()).hexdigest() != t["sha256"]:
        return None
    return t["bytes"]


def rank_cells(rank: int, world: int, limit: int = 0) -> list:
    """Sweep cells solved by `rank` of `world` replicas: cells c with c % world == rank (one
    cell per rank beyond nine ranks); at most `limit` of them when limit > 0."""
    cells = [c for c in range(9) if c % world == rank] or [rank % 9]
    return cells[:limit] if limit > 0 else cells


def max_over_ranks(x: float, dist_mod=None, device="cpu") -> float:
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist_mod is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
    return float(t.item())


def throughput(world: int, solves_per_rank: int, max_ms: float) -> float:
    """Whole-job solves per second: every rank's solves over the slowest rank's time."""
    return world * solves_per_rank / (max_ms / 1000.0)


def workload_desc(n):
    return (f"2D Poisson control, Q1, {n}x{n} nodes, y_d = seeded sum of 8 Gaussians, "
            f"alpha x beta sweep {{1e-2,1e-4,1e-6}} x {{1e-2,1e-3,1e-4}}, u in [-30,30], y <= 0.1, "
            f"kkt_rel <= 1e-6")


def pct(xs, q):
    import numpy as np
    return float(np.percentile(np.asarray(xs, dtype=float), q))


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# the oracle on this host's cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count(), model or "unknown"


def oracle_reference_counts(cell: int):
    """IPM steps and Krylov iterations of the oracle's own full solve of a sweep cell at
    1025^2 (recorded when the oracle wrote the full-size expected values), or None."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"fullsize_poisson2d_1025_cell{cell}.npz")
    if not os.path.exists(path):
        return None
    d = np.load(path)
    return int(d["k"]), int(d["krylov_iters"].sum())


def oracle_sample(cell: int, max_krylov: int, threads: int, n: int = N_DEFAULT,
                  timeout: float = 600.0):
    """Time the oracle (iterative tier: Algorithm A.1 with FGMRES + P_T Newton solves) on its
    first IPM step of one sweep cell, in a child process with `threads` threads (0 = the
    libraries' default, all cores): the QP assembly, the preconditioner construction and
    up to `max_krylov` FGMRES iterations of the first Newton system."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import workloads as W
from oracle import qp as Q, ipm, iterative
wl = W.workload_c2(n={n}, cell={cell})
t0 = time.perf_counter()
qp = Q.from_workload(wl)
t1 = time.perf_counter()
st = []
ipm.solve(qp, sigma=wl.sigma, n_iter=1, common_step=True,
          newton_solve=iterative.newton_solver("gmg", stats=st, maxiter={max_krylov}, accept=1.0))
t2 = time.perf_counter()
print(json.dumps(dict(build_s=t1 - t0, step_s=t2 - t1, setup_s=st[0].setup_s,
                      krylov_s=st[0].solve_s, iters=st[0].iterations, relres=st[0].relres)))
"""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    if threads > 0:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr.strip()[-300:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_solve_seconds(s: dict, counts) -> float:
    """Whole-solve time of the oracle extrapolated from one sample: assembly once, the
    per-IPM-step remainder (preconditioner construction, Theta, right-hand side, update) on
    every step, and the measured time per FGMRES iteration on every iteration of the
    oracle's own full solve of the cell (k IPM steps, K Krylov iterations)."""
    k, K = counts
    per_iter = s["krylov_s"] / max(s["iters"], 1)
    per_step = s["step_s"] - s["krylov_s"]
    return s["build_s"] + k * per_step + K * per_iter


def cpu_baseline(cell: int = 1, max_krylov: int = 0):
    """The oracle on this host's cores at the headline grid: one whole IPM step (its Newton
    system to the FP64 attainable accuracy) of a sweep cell, single-thread and with the
    libraries' default threads; solves/s extrapolated to the oracle's own full solve."""
    counts = oracle_reference_counts(cell)
    cores, model = host_cpu()
    maxk = max_krylov if max_krylov > 0 else 2000
    out = {"unit": "solves/s", "kind": "oracle", "host_cores": cores, "cpu_model": model}
    try:
        one = oracle_sample(cell, maxk, 1)
        allc = oracle_sample(cell, maxk, 0)
    except Exception as e:  # report, do not fail the GPU line
        out.update({"value": None, "cores": 1, "sample": f"failed: {e}"})
        return out
    if counts is None:
        counts = (9, one["iters"] * 9)
    t1 = oracle_solve_seconds(one, counts)
    ta = oracle_solve_seconds(allc, counts)
    out.update({
        "value": 1.0 / t1, "cores": 1,
        "all_cores": {"value": 1.0 / ta, "cores": cores,
                      "measured_step_s": allc["step_s"], "krylov_iters": allc["iters"]},
        "measured": {"qp_assembly_s": one["build_s"], "ipm_step_s": one["step_s"],
                     "precond_setup_s": one["setup_s"], "krylov_s": one["krylov_s"],
                     "krylov_iters": one["iters"], "relres": one["relres"]},
        "extrapolated_solve_s": t1,
        "sample": (f"first IPM step of sweep cell {cell} at {N_DEFAULT}^2 (oracle iterative tier: "
                   f"FGMRES + P_T with its own Galerkin multigrid, Newton system to the FP64 "
                   f"attainable accuracy), single thread; value = 1 / (assembly + {counts[0]} x "
                   f"per-step set-up + {counts[1]} x measured seconds per FGMRES iteration), "
                   f"{counts[0]} IPM steps and {counts[1]} Krylov iterations being the oracle's own "
                   f"full solve of this cell to kkt_rel 1e-6"),
    })
    return out


def run_reference(args, rank, world):
    """Reference arm: the oracle itself on this host's cores, one bounded sample per step:
    the first Newton system of a sweep cell at 1025^2 (rotating over the cells), FGMRES + P_T
    capped at a few iterations; solves/s extrapolated from the measured per-iteration and
    per-step times to the oracle's own full solve."""
    if rank != 0:
        return
    cap = 6
    counts = oracle_reference_counts(1) or (9, 150)
    for k in range(args.warmup):  # warm-up: the QP assembly only
        oracle_sample(k % 9, 1, 1)
    samples = [oracle_sample(k % 9, cap, 1) for k in range(args.steps)]
    per_iter = statistics.mean(s["krylov_s"] / max(s["iters"], 1) for s in samples)
    per_step = statistics.mean(s["step_s"] - s["krylov_s"] for s in samples)
    build = statistics.mean(s["build_s"] for s in samples)
    solve_s = build + counts[0] * per_step + counts[1] * per_iter
    value = 1.0 / solve_s
    cores, model = host_cpu()
    sample = (f"per step: the first Newton system of sweep cell (step mod 9) at {N_DEFAULT}^2, "
              f"oracle iterative tier, FGMRES + P_T capped at {cap} iterations, 1 thread; value "
              f"extrapolated to a whole solve ({counts[0]} IPM steps, {counts[1]} FGMRES "
              f"iterations: the oracle's own full solve of cell 1)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * solve_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(N_DEFAULT), "sample": "bounded, extrapolated"},
            "value_is_extrapolated": True,
            "measured": {"seconds_per_fgmres_iteration": per_iter,
                         "seconds_per_ipm_step_setup": per_step, "qp_assembly_s": build,
                         "sampled_iterations": sum(s["iters"] for s in samples)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "host_cores": cores, "cpu_model": model, "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU path
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import numpy as np
    import torch

    import workloads as W
    from paper_1806_05896_gb300 import ipm

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.n
    stream = torch.cuda.Stream()
    # one solver per sweep cell owned by this rank, inputs resident in HBM
    # args.cells > 0: fewer solvers (smaller device footprint, e.g. for profiler captures)
    cells = rank_cells(rank, world, args.cells)
    solvers, yds, yd_host = {}, {}, {}
    for c in cells:
        wl = W.workload_c2(n=n, cell=c)
        s = ipm.Solver(2, n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
        s.set_stream(stream.cuda_stream)
        yd_host[c] = np.ascontiguousarray(wl.yd)
        yds[c] = torch.as_tensor(yd_host[c].reshape(-1)).cuda()
        s.set_data_device(yds[c])
        solvers[c] = s

    def opts(prec, common=1):
        return ipm.default_options(precision=prec, krylov=ipm.KRYLOV_GMRES_PT, stop=ipm.STOP_KKT,
                                   kkt_tol=1e-6, restart=50, max_krylov=200, common_step=common,
                                   max_ipm=60, kernel_flags=args.kernel_flags)

    def timed(prec, steps, warmup, e2e=False, common=1):
        """`steps` solves after `warmup` untimed ones, rotating over this rank's cells in the
        same order for every leg; whole-region and per-solve CUDA-event times."""
        o = opts(prec, common)
        order = [cells[k % len(cells)] for k in range(warmup + steps)]
        reps = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        u_host = np.empty(n * n)
        for k in range(warmup):
            solvers[order[k]].set_data_device(yds[order[k]])
            solvers[order[k]].solve(o)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = ipm.launch_count()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            t0.record(stream)
            for k in range(steps):
                c = order[warmup + k]
                s = solvers[c]
                ev[k][0].record(stream)
                if e2e:
                    s.set_data(yd_host[c])                 # host -> device inside the step
                    reps.append(s.solve(o))
                    u_host[:] = s.control().reshape(-1)    # device -> host inside the step
                else:
                    s.set_data_device(yds[c])
                    reps.append(s.solve(o))
                ev[k][1].record(stream)
            t1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        launches = ipm.launch_count() - l0
        total_ms = max_over_ranks(t0.elapsed_time(t1), dist, "cuda")
        lat = [a.elapsed_time(b) for a, b in ev]
        return dict(ms=total_ms, lat=lat, reps=reps, launches=launches,
                    cells=order[warmup:])

    def leg_summary(r, steps):
        reps = r["reps"]
        return {"value": throughput(world, steps, r["ms"]), "ms_per_step": r["ms"] / steps,
                "steps": steps,
                "latency_ms": {"p50": pct(r["lat"], 50), "p99": pct(r["lat"], 99)},
                "ipm_iters": statistics.mean(x["ipm_iters"] for x in reps),
                "krylov_iters_per_ipm": statistics.mean(
                    x["krylov_iters_total"] / max(x["ipm_iters"], 1) for x in reps),
                "kkt_rel_max": max(x["kkt_rel"] for x in reps),
                "all_converged": all(x["status"] == ipm.OK for x in reps)}

    K = args.steps
    warm = max(args.warmup, 0)
    with ClockSampler(local) as clk:
        mx = timed(ipm.PREC_MIXED, K, warm)
    clocks = clk.summary()
    if args.legs == "mixed":  # the timed leg only (used for kernel launch lists)
        print(json.dumps({"metric": METRIC, "value": throughput(world, K, mx["ms"]),
                          "unit": "solves/s", "legs": "mixed", "gpu_launches": mx["launches"],
                          "ms_per_step": mx["ms"] / K}))
        return
    # the same cells, the same order: the all-FP64 path and the end-to-end path
    f64 = timed(ipm.PREC_FP64, K, 1)
    e2e = timed(ipm.PREC_MIXED, K, 1, e2e=True)
    # Algorithm A.1 as printed (separate primal and dual step lengths) on the same cells
    sep = timed(ipm.PREC_MIXED, len(cells), 1, common=0)
    kernels = profile_kernels(ipm, solvers, cells, opts(ipm.PREC_MIXED))

    value = throughput(world, K, mx["ms"])
    hbm, peak_kind = measured_peaks()
    mixed = leg_summary(mx, K)
    nodes = (n - 2) ** 2
    kry = sum(x["krylov_iters_total"] for x in mx["reps"])
    agg_gbs = SOLVE_BYTES_PER_NODE_ITER * nodes * kry / (mx["ms"] / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": warm, "ms_per_step": mx["ms"] / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32 (mixed: FP32 multigrid/Chebyshev, FP64 Krylov/IPM)",
        "data": "synthetic",
        "config": {"workload": workload_desc(n), "precision": "mixed", "krylov": "FGMRES + P_T",
                   "ipm": "Algorithm A.1, sigma 0.2, mu0 1, common primal-dual step length",
                   "cells_per_rank": len(cells), "parallelism": f"replicas x{world}",
                   "l2": "per-solve working set (Krylov basis ~3.5 GB) exceeds L2"},
        "latency_ms": mixed["latency_ms"],
        "ipm_iters": mixed["ipm_iters"],
        "krylov_iters_per_ipm": mixed["krylov_iters_per_ipm"],
        "kkt_rel_max": mixed["kkt_rel_max"],
        "fp64": leg_summary(f64, K),
        "mixed_over_fp64": value / leg_summary(f64, K)["value"],
        "separate_step_lengths": separate_summary(sep, leg_summary, ipm),
        "e2e": {"value": throughput(world, K, e2e["ms"]), "unit": "solves/s",
                "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * n * 8,
                "latency_ms": {"p50": pct(e2e["lat"], 50), "p99": pct(e2e["lat"], 99)}},
        "gpu_launches": mx["launches"],
        "launches_per_krylov_iter": mx["launches"] / max(kry, 1),
        "solve_aggregate": {"bytes_per_node_per_krylov_iter": SOLVE_BYTES_PER_NODE_ITER,
                            "achieved_gbs": agg_gbs, "frac_of_hbm": agg_gbs / hbm,
                            "peak": hbm, "peak_kind": peak_kind},
        "roofline": roofline_entry(kernels, hbm, peak_kind),
        "kernels": kernels,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extra:
        line["other_configs"] = other_configs(ipm, W, np)
        line["serving"] = serving(ipm, W, np, args.serve_requests, args.serve_workers)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s in solvers.values():
        s.close()
    if dist:
        dist.destroy_process_group()


def separate_summary(r, leg_summary, ipm):
    """Algorithm A.1 with the printed separate step lengths: per cell, and solves/s over the
    cells where it reaches kkt_rel 1e-6 within 60 IPM steps."""
    rows = []
    for c, rep, ms in zip(r["cells"], r["reps"], r["lat"]):
        rows.append({"cell": c, "converged": rep["status"] == ipm.OK and rep["kkt_rel"] <= 1e-6,
                     "ipm_iters": rep["ipm_iters"], "ms": ms, "kkt_rel": rep["kkt_rel"]})
    ok = [x for x in rows if x["converged"]]
    return {"rule": "alpha_P, alpha_D separate (Algorithm A.1 as printed)",
            "cells": rows,
            "converged_cells": len(ok),
            "solves_per_s_converged": (len(ok) / (sum(x["ms"] for x in ok) / 1000.0)) if ok else None,
            "ipm_iters_converged": statistics.mean(x["ipm_iters"] for x in ok) if ok else None}


def profile_kernels(ipm, solvers, cells, o):
    """CUDA-event timing of the main kernels of the mixed solve (one eager solve each, every
    2nd launch sampled, on the solver's stream): average launch time, launches per solve,
    and algorithmic bytes per launch counted per pass and once."""
    import torch
    out = []
    for kind, name in enumerate(ipm.Solver.KERNELS):
        s = solvers[cells[kind % len(cells)]]
        s.profile_kernel(kind, True, 2)
        s.solve(o)
        torch.cuda.synchronize()
        d = s.profile_kernel_read()
        s.profile_kernel(kind, False)
        if d["sampled"] == 0:
            continue
        avg_s = d["ms"] / d["sampled"] / 1000.0
        out.append({"kernel": name, "avg_launch_us": avg_s * 1e6, "launches_per_solve": d["calls"],
                    "ms_per_solve": avg_s * 1000.0 * d["calls"],
                    "bytes_pass": d["bytes_pass"], "bytes_once": d["bytes_once"],
                    "achieved_gbs_pass": d["bytes_pass"] / avg_s / 1e9,
                    "achieved_gbs_once": d["bytes_once"] / avg_s / 1e9,
                    "sampled_launches": d["sampled"]})
    out.sort(key=lambda x: -x["ms_per_solve"])
    return out


KERNEL_NAMES = {
    "finest_pre_restrict": "k_mg2_pre_restrict_rb<52,52,5,16> (finest level: 5 Jacobi sweeps + "
                           "residual + restriction)",
    "finest_prolong_post": "k_mg2_prolong_post_rb<56,32,5,8> (finest level: prolongation + 5 sweeps)",
    "coarse_cycle": "k_mg2_coarse<float> (one-CTA V-cycle on the levels 65^2 ... 3^2)",
    "saddle_operator": "k_newton_apply_ff2 / k_newton_apply (saddle operator of (NewtonSystem): "
                       "float-float on the Arnoldi path, FP64 for the true residuals)",
    "mid_level_tiles": "k_mg2_pre_restrict_rb<20,32,5,8> / k_mg2_prolong_post_rb<24,24,5,8> "
                       "(levels 513^2 ... 129^2)",
}


def roofline_entry(kernels, hbm, peak_kind):
    """Roofline of the kernel with the most time per solve, its algorithmic bytes per launch
    counted per pass (every sweep reads its operands and writes its result once)."""
    if not kernels:
        return None
    k = kernels[0]
    achieved = k["achieved_gbs_pass"]
    traffic = traffic_if_current(k["kernel"])
    return {"bound": "hbm", "kernel": KERNEL_NAMES.get(k["kernel"], k["kernel"]),
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "peak_kind": peak_kind,
            "algorithmic_bytes_per_launch": k["bytes_pass"],
            "avg_launch_us": k["avg_launch_us"], "sampled_launches": k["sampled_launches"],
            "per_launch_once": {"bytes": k["bytes_once"], "achieved": k["achieved_gbs_once"],
                                "frac": k["achieved_gbs_once"] / hbm},
            "share_of_kernel_time": k["ms_per_solve"] / sum(x["ms_per_solve"] for x in kernels)}


def _timed_solves(ipm, s, o, reps=5):
    import torch
    s.solve(o)  # warm-up (graph capture)
    ms, rep = [], None
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        rep = s.solve(o)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return ms, rep


def other_configs(ipm, W, np):
    """Timed solves of the 513^2 convection-diffusion and 129^3 Poisson configurations, mixed
    precision and FP64."""
    out = {}
    for name, wl in (("cd2d_513_supg", W.workload_c4(n=513)),
                     ("poisson3d_129", W.workload_c3(n=129))):
        s = ipm.Solver(wl.dim, wl.n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb, kind=wl.kind,
                       eps=wl.eps)
        s.set_data(wl.yd)
        res = {}
        for prec, pname in ((ipm.PREC_MIXED, "mixed"), (ipm.PREC_FP64, "fp64")):
            o = ipm.default_options(stop=ipm.STOP_KKT, kkt_tol=1e-6, common_step=1, sigma=wl.sigma,
                                    max_ipm=60, precision=prec, krylov=ipm.KRYLOV_GMRES_PT)
            ms, rep = _timed_solves(ipm, s, o, 5 if pname == "mixed" else 2)
            res[pname] = {"ms_per_solve": statistics.mean(ms), "solves_per_s": 1000.0 / statistics.mean(ms),
                          "p50_ms": pct(ms, 50), "p99_ms": pct(ms, 99), "solves": len(ms),
                          "ipm_iters": rep["ipm_iters"],
                          "krylov_iters_per_ipm": rep["krylov_iters_total"] / max(rep["ipm_iters"], 1),
                          "kkt_rel": rep["kkt_rel"]}
        res["krylov"] = "FGMRES + P_T"
        out[name] = res
        s.close()
    return out


def serving(ipm, W, np, num, workers=16):
    """Seeded request stream (2D 65..513, 3D 33..65, 70/30 Poisson/CD) through the native
    server: a closed-loop burst (saturation throughput), then open loops at 0.8x and 1.5x that
    rate (exponential gaps), p50/p99 latency from submission to completion."""
    reqs = W.serving_stream(num, seed=0)
    opts = dict(precision=ipm.PREC_MIXED, stop=ipm.STOP_KKT, kkt_tol=1e-6, common_step=1,
                max_ipm=60, restart=30)
    sv = ipm.Server(workers=workers, budget_bytes=96 << 30)

    def submit(r, o=opts):
        return sv.submit(r["dim"], r["n"], r["alpha"], r["beta"], r["ua"], r["ub"], r["yd"],
                         kind=r["kind"], eps=r["eps"], sigma=r["sigma"], **o)
    seen = {}
    for r in reqs:  # warm: one request per distinct grid and state equation
        seen.setdefault((r["dim"], r["n"], r["kind"]), r)
    for t in [submit(r) for r in seen.values()]:
        sv.wait(t)
    t0 = time.perf_counter()
    tickets = [submit(r) for r in reqs]
    res = [sv.wait(t) for t in tickets]
    burst_s = time.perf_counter() - t0
    sat = num / burst_s
    out = {"requests": num, "workers": workers,
           "saturation": {"solves_per_s": sat, "p50_ms": 1000 * pct([x[2] for x in res], 50),
                          "p99_ms": 1000 * pct([x[2] for x in res], 99),
                          "converged": sum(x[0]["kkt_rel"] <= 1e-6 for x in res)}}
    for load in (0.8, 1.5):
        gap = 1.0 / (load * sat)
        t0 = time.perf_counter()
        tickets = []
        for r in reqs:
            time.sleep(r["gap"] * gap)
            tickets.append(submit(r))
        lat = [sv.wait(t)[2] for t in tickets]
        dt = time.perf_counter() - t0
        out[f"open_loop_{load}x"] = {"offered_per_s": load * sat, "solves_per_s": num / dt,
                                     "p50_ms": 1000 * pct(lat, 50), "p99_ms": 1000 * pct(lat, 99)}
    # the same stream prefix in mixed precision and all-FP64, closed loop, same server
    head = reqs[:min(num, 128)]
    for name, prec in (("mixed", ipm.PREC_MIXED), ("fp64", ipm.PREC_FP64)):
        o = dict(opts, precision=prec)
        t0 = time.perf_counter()
        res = [sv.wait(t) for t in [submit(r, o) for r in head]]
        dt = time.perf_counter() - t0
        out.setdefault("precision_same_stream", {"requests": len(head)})[name] = {
            "solves_per_s": len(head) / dt,
            "converged": sum(x[0]["kkt_rel"] <= 1e-6 for x in res)}
    sv.close()
    out["mix"] = ("2D {65,129,257,513}^2, 3D {33,65}^3, Poisson/CD 70/30 (CD 2D only), "
                  "log-uniform alpha, beta, Gaussian-sum y_d, mixed precision, kkt_rel 1e-6")
    return out


def sweep_table(sizes, recipe):
    """Iteration counts, solve times and sparsity on several grids.

    recipe "gauss": the 1025^2 benchmark's (alpha, beta) sweep (Gaussian-sum y_d, u in
    [-30, 30], y <= 0.1), FGMRES + P_T, kkt_rel <= 1e-6, common step.
    recipe "poisson": the Poisson table of Section 5.1 (y_d = sin(pi x) sin(pi y),
    u in [-2, 1.5], beta = 1e-2, sigma = 0.2, alpha in {1e-2, 1e-4, 1e-6}), GMRES + P_T and
    MINRES + P_D, the paper's stopping rule (||xi_p||, ||xi_d||, ||xi_c|| <= 1e-6).
    recipe "cd": the convection-diffusion table of Section 5.2 (recirculating wind, SUPG,
    y_d = exp(-64 |x - (1/2, 1/2)|^2), u in [-2, 1.5], beta = 1e-3, eps = 1e-1 (sigma 0.25)
    and 1e-2 (sigma 0.4)), GMRES + P_T, the paper's stopping rule.
    recipe "sparsity": the sparsity table of Section 5.1 (h = 2^-5 when n = 33; the Poisson
    recipe with beta in {1e-1, 1e-2, 1e-3}), GMRES + P_T."""
    import numpy as np
    import torch

    import workloads as W
    from paper_1806_05896_gb300 import ipm

    torch.cuda.set_device(0)
    rows = []

    def run(s, wl, o, extra):
        s.solve(o)  # first solve captures the CUDA graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = s.solve(o)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        u = s.control().reshape(-1)
        interior = np.zeros((wl.n, wl.n), bool)
        interior[1:-1, 1:-1] = True
        u = u[interior.reshape(-1)]
        h = 1.0 / (wl.n - 1)
        every = (np.sum(np.abs(u) < 1e-2) + (wl.n * wl.n - u.size)) / (wl.n * wl.n)
        row = {"n": wl.n, "alpha": wl.alpha, "beta": wl.beta, "ipm_iters": r["ipm_iters"],
               "sparsity_pct_all_nodes": 100.0 * float(every), "u_l1_nodal": float(np.abs(u).sum()),
               "krylov_per_ipm": r["krylov_iters_total"] / max(r["ipm_iters"], 1),
               "ms": dt * 1e3, "kkt_rel": r["kkt_rel"], "status": r["status"],
               "sparsity_pct_interior": 100.0 * float(np.mean(np.abs(u) < 1e-2)),
               "u_l1": h * h * float(np.abs(u).sum())}
        row.update(extra)
        rows.append(row)

    for n in sizes:
        if recipe == "gauss":
            for c in range(9):
                wl = W.workload_c2(n=n, cell=c)
                s = ipm.Solver(2, n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
                s.set_data(wl.yd)
                for prec, name in ((ipm.PREC_MIXED, "mixed"), (ipm.PREC_FP64, "fp64")):
                    o = ipm.default_options(precision=prec, krylov=ipm.KRYLOV_GMRES_PT,
                                            stop=ipm.STOP_KKT, kkt_tol=1e-6, common_step=1,
                                            max_ipm=60)
                    run(s, wl, o, {"precision": name, "krylov": "FGMRES+P_T"})
                s.close()
            continue
        cases = []
        if recipe == "sparsity":
            for a in (1e-2, 1e-4, 1e-6):
                for b in (1e-1, 1e-2, 1e-3):
                    cases.append((W.workload_c1(n=n, alpha=a, beta=b, ua=-2.0, ub=1.5), {}))
        elif recipe == "poisson":
            for a in (1e-2, 1e-4, 1e-6):
                cases.append((W.workload_c1(n=n, alpha=a, beta=1e-2, ua=-2.0, ub=1.5), {}))
        else:
            for eps, sig in ((1e-1, 0.25), (1e-2, 0.4)):
                for a in (1e-2, 1e-4, 1e-6):
                    cases.append((W.workload_c4(n=n, eps=eps, alpha=a, beta=1e-3, sigma=sig),
                                  {"eps": eps}))
        for wl, extra in cases:
            s = ipm.Solver(2, n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb, kind=wl.kind,
                           eps=wl.eps)
            s.set_data(wl.yd)
            krs = ((ipm.KRYLOV_GMRES_PT, "GMRES+P_T"), (ipm.KRYLOV_MINRES_PD, "MINRES+P_D"))
            if recipe == "sparsity":
                krs = krs[:1]
            for kr, kname in krs:
                o = ipm.default_options(precision=ipm.PREC_FP64, krylov=kr, stop=ipm.STOP_PAPER,
                                        sigma=wl.sigma, max_ipm=80, max_krylov=400)
                if kr == ipm.KRYLOV_MINRES_PD and wl.kind == "cd":
                    continue  # P_D with MINRES needs a symmetric saddle matrix
                e = dict(extra)
                e.update({"precision": "fp64", "krylov": kname, "sigma": wl.sigma})
                run(s, wl, o, e)
            s.close()
    print(json.dumps({"sweep_table": rows, "recipe": recipe}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=9)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="all", choices=["all", "mixed"])
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--cells", type=int, default=0, help="sweep cells per rank (0 = all nine)")
    ap.add_argument("--kernel-flags", type=int, default=0,
                    help="ipm_options.kernel_flags of the timed solves (profiler runs pin the "
                         "tile shapes with 512: timings under a profiler mislead the autotuner)")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-workers", type=int, default=16)
    ap.add_argument("--sweep-table", default="",
                    help="comma-separated grid sizes: print a sweep table and exit")
    ap.add_argument("--recipe", default="gauss", choices=["gauss", "poisson", "cd", "sparsity"])
    args = ap.parse_args()
    if args.sweep_table:
        sweep_table([int(v) for v in args.sweep_table.split(",")], args.recipe)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()

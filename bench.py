"""Benchmark: interior point solves per second on the 1025^2 Poisson control sweep.

One step = one complete solve (Algorithm A.1 with preconditioned Krylov Newton
solves, every stage in libipm's CUDA kernels) of one cell of the sweep
alpha in {1e-2, 1e-4, 1e-6} x beta in {1e-2, 1e-3, 1e-4} (steps rotate over the
nine cells), Gaussian-sum y_d, u in [-30, 30], y <= 0.1, stopped at relative KKT
residual 1e-6. The headline value uses the mixed-precision path; the all-FP64
path is measured beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own share of the sweep (replicas,
no collective on the data path); value = all solves / max-over-ranks time.
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

# DRAM traffic per launch of the roofline kernel (finest level of the 1025^2 grid) from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, profiles/ summary named
# below), valid while the kernel's source region is unchanged (hash checked at run time).
ROOF_KERNEL = "k_mg2_pre_restrict_rb<52,52,5,16> (finest level: 5 Jacobi sweeps + residual + restriction)"
ROOF_TRAFFIC = {"bytes": 8406272,
                "sha256": "9a64e0b6708af13123b538ab508c4a54c6378464e9457538b8c4224f88750625",
                "profile": "profiles/mg2_pre_restrict_rb_1025_full.md"}
ROOF_SRC = ("paper_1806_05896_gb300/csrc/k_mg_fused.cu",
            "// Register-blocked FP32 tile kernels",
            "__global__ void __launch_bounds__(NW * 32) k_mg2_prolong_post_rb")


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


def roof_source_hash():
    import hashlib
    with open(os.path.join(ROOT, ROOF_SRC[0])) as f:
        src = f.read()
    i, j = src.find(ROOF_SRC[1]), src.find(ROOF_SRC[2])
    return hashlib.sha256(src[i:j].encode()).hexdigest() if 0 <= i < j else None
N_DEFAULT = 1025
SAMPLE_N = 129  # oracle sample grid for the CPU baseline


def workload_desc(n):
    return (f"2D Poisson control, Q1, {n}x{n} nodes, y_d = seeded sum of 8 Gaussians, "
            f"alpha x beta sweep {{1e-2,1e-4,1e-6}} x {{1e-2,1e-3,1e-4}}, u in [-30,30], y <= 0.1, "
            f"kkt_rel <= 1e-6")


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


# ---------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def cpu_baseline(steps_desc: str, cell: int = 0, timeout: float = 120.0):
    """The oracle (scipy sparse-direct Algorithm A.1) timed on this host, in a child process."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import workloads as W
from oracle import qp as Q, ipm
wl = W.workload_c2(n={SAMPLE_N}, cell={cell})
t = time.perf_counter()
qp = Q.from_workload(wl)
r = ipm.solve(qp, sigma=wl.sigma, stop="kkt", kkt_tol=1e-6, common_step=True)
dt = time.perf_counter() - t
print(json.dumps(dict(seconds=dt, iters=len(r.history) - 1, kkt=r.history[-1]["kkt_rel"])))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=timeout)
    if r.returncode != 0:
        return {"value": None, "unit": "solves/s", "cores": 1, "kind": "oracle",
                "sample": f"failed: {r.stderr.strip()[-200:]}"}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    scale = ((SAMPLE_N - 2) ** 2) / ((N_DEFAULT - 2) ** 2)
    return {"value": scale / d["seconds"], "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"one full oracle solve of sweep cell {cell} at {SAMPLE_N}^2 nodes "
                       f"({d['iters']} IPM steps, {d['seconds']:.2f} s, sparse-direct Newton solves, "
                       f"1 thread); value scaled to 1025^2 by the unknown-count ratio {scale:.4g} "
                       f"(optimistic for the oracle, whose factorisation grows faster than linearly)"),
            "seconds": d["seconds"]}


def run_reference(args, rank, world):
    """Reference arm: the oracle itself, one sampled solve per step, on this host's cores."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline("warmup")
    samples = [cpu_baseline("step", cell=k % 9) for k in range(args.steps)]
    ok = [c for c in samples if c["value"]]
    scale = ((SAMPLE_N - 2) ** 2) / ((N_DEFAULT - 2) ** 2)
    # solves per second at 1025^2 over the timed samples (each scaled by the unknown ratio)
    scaled_s = [c["seconds"] / scale for c in ok]
    value = len(scaled_s) / sum(scaled_s) if scaled_s else None
    cb = {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
          "sample": (f"{len(ok)} full oracle solves of sweep cells 0..{min(args.steps, 9) - 1} "
                     f"at {SAMPLE_N}^2 nodes (sparse-direct Newton solves, 1 thread), "
                     f"{statistics.mean(c['seconds'] for c in ok):.2f} s each on average; "
                     f"scaled to 1025^2 by the unknown-count ratio {scale:.4g}") if ok else
                    "failed"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(scaled_s) if scaled_s else None,
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(N_DEFAULT), "sample_grid": SAMPLE_N},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    def opts(prec):
        return ipm.default_options(precision=prec, krylov=ipm.KRYLOV_GMRES_PT, stop=ipm.STOP_KKT,
                                   kkt_tol=1e-6, restart=50, max_krylov=200, common_step=1,
                                   max_ipm=60)

    def timed(prec, steps, warmup, e2e=False, profile=False):
        o = opts(prec)
        order = [cells[k % len(cells)] for k in range(warmup + steps)]
        lat, reps = [], []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        u_host = np.empty(n * n)
        for k in range(warmup):
            solvers[order[k]].solve(o)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        if profile:
            for s in solvers.values():
                s.profile_smoother(True, 4)
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
        prof = None
        if profile:
            tot, cnt, by = 0.0, 0, 0.0
            for s in solvers.values():
                ms, c_, b_ = s.profile_read()
                tot += ms
                cnt += c_
                by = b_
                s.profile_smoother(False, 4)
            prof = (tot, cnt, by)
        return total_ms, lat, reps, launches, prof

    warm = max(args.warmup, 0)
    with ClockSampler(local) as clk:
        tot_mx, lat_mx, reps_mx, launches, _ = timed(ipm.PREC_MIXED, args.steps, warm)
    clocks = clk.summary()
    if args.legs == "mixed":  # the timed leg only (used for kernel launch lists)
        print(json.dumps({"metric": METRIC, "value": throughput(world, args.steps, tot_mx),
                          "unit": "solves/s", "legs": "mixed", "gpu_launches": launches}))
        return
    # dominant kernel: finest-level multigrid smoothing launches timed by CUDA events on the
    # solver stream during one more solve per cell (eager launches: events cannot sit
    # inside the replayed graphs of the timed region)
    _, _, _, _, prof = timed(ipm.PREC_MIXED, min(len(cells), 3), 0, profile=True)
    fp64_steps = max(1, min(args.steps, 3))
    tot_64, lat_64, reps_64, _, _ = timed(ipm.PREC_FP64, fp64_steps, 1)
    tot_e2e, lat_e2e, _, _, _ = timed(ipm.PREC_MIXED, max(1, min(args.steps, 5)), 1, e2e=True)

    K = args.steps
    value = throughput(world, K, tot_mx)
    pct = lambda xs, q: float(np.percentile(np.asarray(xs), q))
    hbm, peak_kind = measured_peaks()
    roof = None
    if prof and prof[1] > 0:
        avg_s = prof[0] / prof[1] / 1000.0
        achieved = prof[2] / avg_s / 1e9
        traffic = None
        if ROOF_TRAFFIC["bytes"] and ROOF_TRAFFIC["sha256"] == roof_source_hash():
            traffic = ROOF_TRAFFIC["bytes"]
        roof = {"bound": "hbm", "kernel": ROOF_KERNEL,
                "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "peak_kind": peak_kind, "sampled_launches": prof[1],
                "avg_launch_us": avg_s * 1e6, "algorithmic_bytes_per_launch": prof[2],
                "note": "largest HBM-streaming kernel; the largest single kernel by time is "
                        "the one-CTA coarse V-cycle (latency-bound on one SM by design)"}
    kkt_max = max(r["kkt_rel"] for r in reps_mx)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": warm, "ms_per_step": tot_mx / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32 (mixed: FP32 multigrid/Chebyshev, FP64 Krylov/IPM)",
        "data": "synthetic",
        "config": {"workload": workload_desc(n), "precision": "mixed", "krylov": "FGMRES + P_T",
                   "ipm": "Algorithm A.1, sigma 0.2, mu0 1, common primal-dual step length",
                   "cells_per_rank": len(cells), "parallelism": f"replicas x{world}",
                   "l2": "per-solve working set (Krylov basis ~3.5 GB) exceeds L2"},
        "latency_ms": {"p50": pct(lat_mx, 50), "p99": pct(lat_mx, 99)},
        "ipm_iters": statistics.mean(r["ipm_iters"] for r in reps_mx),
        "krylov_iters_per_ipm": statistics.mean(r["krylov_iters_total"] / max(r["ipm_iters"], 1)
                                                for r in reps_mx),
        "kkt_rel_max": kkt_max,
        "fp64": {"value": throughput(world, fp64_steps, tot_64), "ms_per_step": tot_64 / fp64_steps,
                 "ipm_iters": statistics.mean(r["ipm_iters"] for r in reps_64),
                 "krylov_iters_per_ipm": statistics.mean(r["krylov_iters_total"] / max(r["ipm_iters"], 1)
                                                         for r in reps_64),
                 "steps": fp64_steps, "latency_ms": {"p50": pct(lat_64, 50), "p99": pct(lat_64, 99)},
                 "kkt_rel_max": max(r["kkt_rel"] for r in reps_64)},
        "e2e": {"value": throughput(world, len(lat_e2e), tot_e2e), "unit": "solves/s",
                "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * n * 8},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extra:
        line["other_configs"] = other_configs(ipm, W, np, stream)
        line["serving"] = serving(ipm, W, np, args.serve_requests)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline("ours")
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s in solvers.values():
        s.close()
    if dist:
        dist.destroy_process_group()


def _timed_solve(ipm, s, o, reps=2):
    import torch
    s.solve(o)  # warm-up (graph capture)
    ms = []
    rep = None
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        rep = s.solve(o)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return min(ms), rep


def other_configs(ipm, W, np, stream):
    """One timed solve each of the 513^2 convection-diffusion and 129^3 Poisson configurations."""
    out = {}
    for name, wl, kw in (("cd2d_513_supg", W.workload_c4(n=513), dict(precision=ipm.PREC_MIXED)),
                         ("poisson3d_129", W.workload_c3(n=129), dict(precision=ipm.PREC_MIXED))):
        s = ipm.Solver(wl.dim, wl.n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb, kind=wl.kind,
                       eps=wl.eps)
        s.set_data(wl.yd)
        o = ipm.default_options(stop=ipm.STOP_KKT, kkt_tol=1e-6, common_step=1, sigma=wl.sigma,
                                max_ipm=60, **kw)
        ms, rep = _timed_solve(ipm, s, o)
        out[name] = {"ms_per_solve": ms, "solves_per_s": 1000.0 / ms, "ipm_iters": rep["ipm_iters"],
                     "krylov_iters_per_ipm": rep["krylov_iters_total"] / max(rep["ipm_iters"], 1),
                     "kkt_rel": rep["kkt_rel"], "precision": "mixed", "krylov": "FGMRES + P_T"}
        s.close()
    return out


def serving(ipm, W, np, num):
    """Seeded request stream (2D 65..513, 3D 33..65, 70/30 Poisson/CD) through the native
    server: a closed-loop burst (saturation throughput) and an open loop at 0.8x that rate."""
    reqs = W.serving_stream(num, seed=0)
    opts = dict(precision=ipm.PREC_MIXED, stop=ipm.STOP_KKT, kkt_tol=1e-6, common_step=1,
                max_ipm=60, restart=30)
    sv = ipm.Server(workers=4, budget_bytes=96 << 30)

    def submit(r):
        return sv.submit(r["dim"], r["n"], r["alpha"], r["beta"], r["ua"], r["ub"], r["yd"],
                         kind=r["kind"], eps=r["eps"], sigma=r["sigma"], **opts)
    seen = {}
    for r in reqs:  # warm: one request per distinct grid and state equation
        seen.setdefault((r["dim"], r["n"], r["kind"]), r)
    for t in [submit(r) for r in seen.values()]:
        sv.wait(t)
    t0 = time.perf_counter()
    tickets = [submit(r) for r in reqs]
    lat = [sv.wait(t)[2] for t in tickets]
    burst_s = time.perf_counter() - t0
    sat = num / burst_s
    gap = 1.0 / (0.8 * sat)
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        time.sleep(r["gap"] * gap)
        tickets.append(submit(r))
    lat2 = [sv.wait(t)[2] for t in tickets]
    open_s = time.perf_counter() - t0
    sv.close()
    pct = lambda xs, q: float(np.percentile(np.asarray(xs), q)) * 1000.0
    return {"requests": num, "workers": 4,
            "saturation": {"solves_per_s": sat, "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99)},
            "open_loop_0.8x": {"offered_per_s": 0.8 * sat, "solves_per_s": num / open_s,
                               "p50_ms": pct(lat2, 50), "p99_ms": pct(lat2, 99)},
            "mix": "2D {65,129,257,513}^2, 3D {33,65}^3, Poisson/CD 70/30 (CD 2D only), "
                   "log-uniform alpha, beta, Gaussian-sum y_d, mixed precision, kkt_rel 1e-6"}


def sweep_table(sizes):
    """The (alpha, beta) sweep on several grids: iteration counts, solve times, sparsity."""
    import numpy as np
    import torch

    import workloads as W
    from paper_1806_05896_gb300 import ipm

    torch.cuda.set_device(0)
    rows = []
    for n in sizes:
        interior = np.zeros((n, n), bool)
        interior[1:-1, 1:-1] = True
        interior = interior.reshape(-1)
        for c in range(9):
            wl = W.workload_c2(n=n, cell=c)
            s = ipm.Solver(2, n, wl.alpha, wl.beta, wl.ua, wl.ub, wl.ya, wl.yb)
            s.set_data(wl.yd)
            for prec, name in ((ipm.PREC_MIXED, "mixed"), (ipm.PREC_FP64, "fp64")):
                o = ipm.default_options(precision=prec, krylov=ipm.KRYLOV_GMRES_PT,
                                        stop=ipm.STOP_KKT, kkt_tol=1e-6, common_step=1,
                                        max_ipm=60)
                s.solve(o)  # first solve captures the CUDA graphs
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = s.solve(o)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                u = s.control().reshape(-1)[interior]
                h = 1.0 / (n - 1)
                rows.append({"n": n, "alpha": wl.alpha, "beta": wl.beta, "precision": name,
                             "ipm_iters": r["ipm_iters"],
                             "krylov_per_ipm": r["krylov_iters_total"] / max(r["ipm_iters"], 1),
                             "ms": dt * 1e3, "kkt_rel": r["kkt_rel"],
                             "sparsity_pct": 100.0 * float(np.mean(np.abs(u) < 1e-2)),
                             "u_l1": h * h * float(np.abs(u).sum())})
            s.close()
    print(json.dumps({"sweep_table": rows}), flush=True)


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
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--sweep-table", default="",
                    help="comma-separated grid sizes: print the (alpha, beta) sweep table and exit")
    args = ap.parse_args()
    if args.sweep_table:
        sweep_table([int(v) for v in args.sweep_table.split(",")])
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()

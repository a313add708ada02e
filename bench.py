"""Benchmark: mixed-precision tile-Cholesky Gaussian log-likelihood on one B300.

Workload (one step = one evaluation of Eq. 2, all of generation, Algorithm 1,
log-determinant and solve): n = 40,000 locations on a 200 x 200 jittered grid
(seed 0) in Morton order, Matern sigma2 = 1, beta = 0.1, nu = 0.5, tile 500,
FP64 band of `--band` tiles, off-band updates as FP32-accurate fixed-point
slice products on the tensor cores (FP16 planes of an 8/12/12-bit split), in-band
updates as FP64-accurate products of seven 8-bit BF16 slices.  Inputs are synthetic (measurements from a seeded spectral
Matern-field simulation).  The working set (3.3 GB of tiles) is far larger than
L2, so consecutive steps do not hit in L2.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
plain FP64 numpy/LAPACK definition of Eq. 2) on a bounded sample of the same
workload instead, under the same metric.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M_GRID = 200          # 200 x 200 = 40,000 locations
NB = 500
THETA = (1.0, 0.1, 0.5, 0.0)
CPU_SAMPLE_M = 100           # oracle sample: 100 x 100 = 10,000 locations (dense FP64 definition)
CPU_ALG1_M = 80              # and 80 x 80 = 6,400 locations for the oracle's Algorithm 1 (tile 400, band 1)
METRIC = "MP tile-Cholesky TFLOP/s (n^3/3 per log-likelihood evaluation); evals/s vs all-FP64 GPU path"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--band", type=int, default=1)
    ap.add_argument("--lp", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the all-FP64 comparison evaluation")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-sweep", action="store_true", help="skip the band sweep (bands 2, 4, 8)")
    ap.add_argument("--no-dmma", action="store_true", help="skip the all-FP64 FP64-pipe (DMMA) comparison (22 s)")
    ap.add_argument("--gen64", action="store_true", help="generate off-band entries in FP64 and round")
    ap.add_argument("--dmma", action="store_true",
                    help="in-band (FP64) updates on the FP64 pipe instead of FP64-accurate tensor-core products")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-evaluation measurement")
    ap.add_argument("--no-dst", action="store_true", help="skip the DST / IND approximation timings")
    ap.add_argument("--no-far", action="store_true", help="skip the far-tier (three-precision) sweep")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-window", type=float, default=3.0, help="seconds of Poisson arrivals served")
    return ap.parse_args()


def max_over_ranks(ms, world, dev):
    """The slowest rank's time of the timed region (every rank holds the same
    number of independent evaluations: replicas)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ms, world, steps, flops_per_eval):
    """Whole-job evals/s and TFLOP/s: the evaluations of all ranks over the
    slowest rank's time."""
    sec = ms / 1000.0
    return world * steps / sec, world * flops_per_eval * steps / sec / 1e12


def shard_problems(costs, rank, world):
    """Indices of the independent problems this rank evaluates: greedy by cost
    (largest first, to the least loaded rank, ties to the lower rank), so the
    ranks' shares are disjoint, cover every problem and have near-equal work."""
    load = [0.0] * world
    mine = []
    for b in sorted(range(len(costs)), key=lambda q: (-costs[q], q)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += costs[b]
        if r == rank:
            mine.append(b)
    return sorted(mine)


def gather_shards(local, world):
    """The per-rank batch results of a sharded run, gathered on every rank:
    (ms of the slowest rank, every problem's completion ms, problems done)."""
    if world <= 1:
        return local["ms"], list(local["completion_ms"]), local["problems"]
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, local)
    return (max(p["ms"] for p in parts), [c for p in parts for c in p["completion_ms"]],
            sum(p["problems"] for p in parts))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(m=M_GRID, seed=0):
    from paper_2003_05324_b300 import inputs
    x, y = inputs.jittered_grid(m, seed=seed)
    z = inputs.matern_field_rff(x, y, THETA[0], THETA[1], THETA[2], seed=seed + 1)
    return x, y, z


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _host_cores():
    try:
        from threadpoolctl import threadpool_info
        return max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        return os.cpu_count()


def cpu_baseline(steps=1, alg1=False):
    """The oracle as it stands on the host cores (numpy/scipy/LAPACK, BLAS
    threads): the dense FP64 definition of Eq. 2 on a bounded sample of the
    workload (alg1=True: the oracle's Algorithm 1 with FP32 tiles instead)."""
    from oracle import geo_oracle as O
    m = CPU_ALG1_M if alg1 else CPU_SAMPLE_M
    x, y, z = workload(m, seed=0)
    perm = O.morton_order(x, y)
    x, y, z = x[perm], y[perm], z[perm]
    th = O.Theta(*THETA)
    n = len(z)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        if alg1:
            O.loglik_mp(x, y, z, th, nb=400, band=1)
        else:
            O.loglik_dense(x, y, z, th)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    what = ("oracle Algorithm 1 (numpy/scipy, FP32 off-band tiles), tile 400, band 1" if alg1 else
            "oracle dense FP64 definition (scipy Matern entries, LAPACK dpotrf, triangular solve)")
    return {"value": n ** 3 / 3.0 / t / 1e12, "unit": "TFLOP/s", "cores": _host_cores(), "kind": "oracle",
            "sample": f"{what} on n={n} ({m}x{m} jittered grid, Morton order), same theta: a bounded sample of "
                      f"the n=40000 workload (the full size needs ~50 GB of host memory for the dense matrix); "
                      f"{t:.2f} s per evaluation, TFLOP/s counted as n^3/3",
            "n": n, "seconds_per_eval": t}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(1)
    t0 = time.perf_counter()
    vals = [cpu_baseline(1) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    v = statistics.median([c["value"] for c in vals])
    cb = dict(vals[0])
    cb["value"] = v
    n = CPU_SAMPLE_M ** 2
    print(json.dumps({
        "impl": "reference", "metric": METRIC,
        "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"loglik n={n} ({CPU_SAMPLE_M}x{CPU_SAMPLE_M} jittered grid, Morton), Matern "
                               f"sigma2=1 beta=0.1 nu=0.5: the dense FP64 oracle on a bounded sample of the "
                               f"n=40000 workload", "n": n,
                   "cache": "inputs larger than L2 not applicable (CPU)"},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


FP64_MEASURED_TFLOPS = 0.97  # DMMA, measured by a one-off microbenchmark on a B300
FP32_MEASURED_TFLOPS = 68.9  # FFMA, same microbenchmark
TC_PAIRS = 6                 # FP16 slice products per off-band update (persistent DAG kernel)
TC_PAIRS_STEPWISE = 10       # BF16 slice products per off-band update (step-by-step kernel)
EX_PAIRS = 28                # BF16 slice products per FP64-accurate in-band update

# DRAM bytes (read + write) of one launch of the factorization kernel on this
# workload (n = 40,000, tile 500, band 1, default flags), keyed by a hash of the
# kernel's sources: a changed kernel reports null.  The figure is scaled from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the same
# kernel at n = 25,600 (p = 52) by the number of off-band tile updates
# (p (p^2 - 1) / 6: 23,426 there, 85,320 here): 3.380 MB per update.  The
# per-update figure falls slowly with size (3.71 / 3.57 / 3.38 MB at
# p = 13 / 29 / 52), so this slightly overstates the full-size traffic.
DAG_SOURCES = ("dag.cu", "dag.cuh", "tc_common.cuh", "geo_internal.cuh", "ysolve.cuh")
DAG_TRAFFIC = {"bd050c17c86bdaab": (46108520960 + 33065969408) / 23426 * 85320}


def dag_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in DAG_SOURCES:
        with open(os.path.join(ROOT, "paper_2003_05324_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def algorithmic_flops(p, nb, band):
    """Algorithmic work of one factorization by kind (Algorithm 1's tasks with
    their textbook counts): FP64 potrf + in-band trsm, FP64 in-band updates
    (dsyrk nb^3, dgemm 2 nb^3), FP32 off-band trsm, off-band sgemm (2 nb^3)."""
    f64 = p * nb ** 3 / 3.0
    f64u = 0.0
    f32 = 0.0
    lp = 0.0
    for k in range(p):
        for i in range(k + 1, p):
            if i - k < band:
                f64 += nb ** 3
            else:
                f32 += nb ** 3
        for j in range(k + 1, p):
            f64u += nb ** 3                      # dsyrk on (j, j), lower triangle
            for i in range(j + 1, p):
                if i - j < band:
                    f64u += 2.0 * nb ** 3
                else:
                    lp += 2.0 * nb ** 3
    return f64, f64u, f32, lp


def tensor_work_band1(n, nb):
    """Algorithmic tensor-core work (BF16-rate flops) of one band-1
    factorization with the in-band updates on the tensor cores, in closed form
    (the counts of algorithmic_flops at band 1): p (p - 1) / 2 dsyrk of nb^3
    flops at EX_PAIRS products and C(p, 3) off-band updates of 2 nb^3 at
    TC_PAIRS products."""
    p = -(-n // nb)
    return (p * (p - 1) / 2.0) * nb ** 3 * EX_PAIRS + (p * (p - 1) * (p - 2) / 6.0) * 2.0 * nb ** 3 * TC_PAIRS


def measured_hbm_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)).get("hbm_gbs", 6400.0), "measured (MEASURED_PEAKS.json)"
    return 6400.0, "fallback (6.4 TB/s of the profiling recipe)"


def tile_mix_roofline(rows, ts, ms_step):
    """The tile-mix-weighted lower bound of one evaluation, with the units taken
    one after another: T* = sum over units of F_unit / P_unit (FP64 pipe, FP32
    pipe, tensor cores, as in the kernel row) + B_gen / BW + B_solve / BW, where
    B_gen = B_solve = the stored tile bytes (written once by the generation,
    read once by the solve) and BW the measured HBM bandwidth.  The persistent
    kernel overlaps the units, so the largest single term is also reported."""
    dag = next((r for r in rows if r["kernel"].startswith("dag_kernel")), None)
    if dag is None:
        return None
    bw, bw_src = measured_hbm_gbs()
    stored = float(ts.lay.bytes_dp + ts.lay.bytes_sp)
    units = dict(dag["unit_lower_bounds_ms"])
    units["HBM (generation writes, solve reads the stored tiles)"] = 2.0 * stored / (bw * 1e9) * 1e3
    t_star = sum(units.values())
    return {"t_star_ms": t_star, "frac": t_star / ms_step, "terms_ms": units, "stored_tile_bytes": stored,
            "largest_term_ms": max(units.values()), "hbm_source": bw_src}


def generation_row(ts, kern5):
    """Roofline row of the covariance generation (Eq. 1): every stored lower
    tile written once in its own precision (FP64 band, FP32 beyond), bound by
    HBM writes for the closed-form nu = 1/2; achieved = those bytes / the
    launch's CUDA-event time."""
    gms, gn = kern5
    if not gn:
        return None
    nb, p, band = ts.nb, ts.p, ts.band
    ndp = sum(1 for j in range(p) for i in range(j, p) if i - j < band)
    nsp = p * (p + 1) // 2 - ndp
    written = float(nb * nb * (8 * ndp + 4 * nsp))
    bw, src = measured_hbm_gbs()
    t = gms / gn / 1000.0
    ach = written / t / 1e9
    return {"kernel": "matern_tiles_kernel (Eq. 1, each tile in its own precision)", "bound": "hbm",
            "achieved": ach, "peak": bw, "unit": "GB/s", "frac": ach / bw, "bytes_per_launch": written,
            "avg_ms": gms / gn, "launches": gn, "total_ms": gms, "peak_source": src}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        pk = json.load(open(path))
        return pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")), "measured (sustained, MEASURED_PEAKS.json)"
    return 1400.0, "fallback (sustained 1.4 PFLOP/s of the profiling recipe)"


def kernel_rows(ts, args, kern):
    """Roofline rows for the factorization kernels timed live in the region.
    The persistent DAG kernel runs every unit at once, so its bound is the
    largest of the per-unit lower bounds F_unit / P_unit; achieved = that
    unit's algorithmic flops / the kernel's measured time."""
    steps = args.steps
    f64, f64u, f32, lp = algorithmic_flops(ts.p, NB, ts.band)
    bf16_peak, bf16_src = measured_peaks()
    ex = args.lp == "bf16" and not args.dmma      # in-band updates on the tensor cores
    tc = lp * TC_PAIRS if args.lp == "bf16" else 0.0
    if ex:
        tc += f64u * EX_PAIRS
    else:
        f64 += f64u
    units = [("FP64 pipe (potrf, in-band trsm" + ("" if ex else ", dsyrk, in-band dgemm") + ")", f64,
              FP64_MEASURED_TFLOPS, "alu", "FP64 DMMA measured by a microbenchmark (0.97 TFLOP/s)"),
             ("FP32 pipe (off-band trsm)", f32 + (lp if args.lp != "bf16" else 0.0), FP32_MEASURED_TFLOPS, "alu",
              "FP32 FFMA measured by a microbenchmark (68.9 TFLOP/s)")]
    if tc:
        units.append(("tensor cores (off-band FP16 slices x %d%s)" % (
                      TC_PAIRS, ", in-band FP64-accurate x %d" % EX_PAIRS if ex else ""), tc, bf16_peak, "tensor",
                      "bf16 " + bf16_src))
    rows = []
    dag_ms, dag_n = kern[4]
    if dag_n:
        t = dag_ms / 1000.0 / steps
        lb = [(f / (pk * 1e12), name, f, pk, bound, src) for name, f, pk, bound, src in units]
        tstar, name, f, pk, bound, src = max(lb)
        ach = f / t / 1e12
        rows.append({"kernel": "dag_kernel (persistent tile DAG: potrf, trsm, dsyrk/dgemm, tcgen05 sgemm)",
                     "bound": bound, "binding_unit": name, "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                     "frac": ach / pk, "lower_bound_ms": tstar * 1e3, "avg_ms": dag_ms / dag_n,
                     "launches": dag_n, "total_ms": dag_ms, "peak_source": src,
                     "unit_lower_bounds_ms": {u[1]: u[0] * 1e3 for u in lb}})
    names = {0: ("fp64_update (dsyrk+dgemm, DMMA)", f64u, FP64_MEASURED_TFLOPS, "alu",
                 "FP64 DMMA measured by a microbenchmark"),
             1: ("offband_update (split-BF16 tcgen05)", lp * TC_PAIRS_STEPWISE, bf16_peak, "tensor",
                 "bf16 " + bf16_src)}
    for kind, (name, f, pk, bound, src) in names.items():
        kms, kn = kern[kind]
        if kn and f:
            ach = f * steps / (kms / 1000.0) / 1e12
            rows.append({"kernel": name, "bound": bound, "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                         "frac": ach / pk, "avg_ms": kms / kn, "launches": kn, "total_ms": kms,
                         "peak_source": src})
    dominant = max(rows, key=lambda r: r["total_ms"]) if rows else None
    roofline = None
    if dominant:
        roofline = {k: dominant[k] for k in ("bound", "achieved", "peak", "unit", "frac")}
        roofline["kernel"] = dominant["kernel"]
        roofline["traffic"] = None
        if dominant["kernel"].startswith("dag_kernel") and ts.n == M_GRID ** 2 and ts.band == 1 and \
                args.lp == "bf16" and not (args.dmma or args.gen64):
            t = DAG_TRAFFIC.get(dag_source_hash())
            roofline["traffic"] = t
            roofline["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel build "
                                          "at n=25600, scaled by the off-band update count (85320 / 23426)"
                                          if t is not None else "no capture of this kernel build")
    return rows, roofline


def batch_workload(geo, dev, nprob=256):
    """256 independent datasets (seed 100 + i): n ~ U[500, 8000] jittered-uniform
    locations, sigma2 ~ U[0.5, 2], beta ~ U[0.02, 0.3], nu in {1/2, 1, 3/2};
    measurements are white noise (the throughput does not depend on them)."""
    import torch
    from paper_2003_05324_b300 import inputs
    rng = np.random.default_rng(100)
    probs, thetas = [], []
    for b in range(nprob):
        n = int(rng.integers(500, 8001))
        th = geo.Theta(float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.02, 0.3)), float(rng.choice([0.5, 1.0, 1.5])))
        x, y = inputs.uniform_points(n, seed=100 + b)
        perm = geo.morton_order(x, y)
        x, y = x[perm], y[perm]
        z = inputs.white_noise(n, seed=1000 + b)
        probs.append(dict(x=torch.as_tensor(x, device=dev), y=torch.as_tensor(y, device=dev),
                          z=torch.as_tensor(z, device=dev)))
        thetas.append(th)
    return probs, thetas


def time_batch(geo, B, thetas, reps, dev):
    """Graph-captured evaluations of batch B: (ms per replay by CUDA events,
    the results of the last one, each problem's completion in ms after the
    factorization launch started, from the launch's own %globaltimer stamps)."""
    import torch
    B.set_theta(thetas)
    B.loglik_async()
    torch.cuda.synchronize(dev)
    B.capture()
    ms, done = [], None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        B.graph.replay()
        e1.record()
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
        done = B.completion_ms()
    return ms, B.out.cpu().numpy(), done


BATCH_BAND_LADDER = (1, 4, 16, 10 ** 6)   # band tried for a problem that is not positive definite at the previous


def run_batch(geo, dev, rank=0, world=1):
    """Batched evaluation: the autotuner times one graph-captured evaluation per
    tile size in {64, 128, 256} (band 1) and keeps the fastest; each problem
    that is not positive definite in mixed precision at one band is re-evaluated
    at the next band of BATCH_BAND_LADDER (more tiles in FP64; the last is all
    FP64) in a follow-up batch, so every problem gets the narrowest band that
    factors it."""
    import torch
    probs, thetas = batch_workload(geo, dev)
    nall = len(probs)
    flops = sum(int(pr["z"].shape[0]) ** 3 / 3.0 for pr in probs)
    if world > 1:   # independent problems: each rank a disjoint, cost-balanced share
        mine = shard_problems([int(pr["z"].shape[0]) ** 3 for pr in probs], rank, world)
        probs, thetas = [probs[b] for b in mine], [thetas[b] for b in mine]
    tune = {}
    for nb in (64, 128, 256):
        B = geo.Batch([dict(pr, nb=nb, band=1) for pr in probs], device=dev)
        ms, _, _ = time_batch(geo, B, thetas, 1, dev)
        tune[nb] = ms[0]
        del B
        torch.cuda.empty_cache()
    nb = min(tune, key=tune.get)
    todo = list(range(len(probs)))
    band_of, stages, t_total, completion = {}, [], 0.0, np.full(len(probs), np.nan)
    for band in BATCH_BAND_LADDER:
        if not todo:
            break
        B = geo.Batch([dict(probs[b], nb=nb, band=band) for b in todo], device=dev)
        ms, out, done = time_batch(geo, B, [thetas[b] for b in todo], 5 if band == 1 else 3, dev)
        del B
        torch.cuda.empty_cache()
        ok = [q for q in range(len(todo)) if np.isfinite(out[q, 0])]
        for q in ok:
            band_of[todo[q]] = band
            completion[todo[q]] = t_total + done[q]
        stages.append({"band": band if band < 10 ** 6 else "all FP64", "problems": len(todo), "factored": len(ok),
                       "ms": statistics.median(ms), "p99_ms": max(ms)})
        if band == 1 and ok:
            # tensor roofline of the band-1 launch: the factored problems'
            # algorithmic tensor work over the time from the launch's start to
            # the last of their completions (the failed ones' partial work is
            # not counted: a lower bound on the achieved rate)
            work = sum(tensor_work_band1(int(probs[todo[q]]["z"].shape[0]), nb) for q in ok)
            t_dag = max(done[q] for q in ok) / 1000.0
            pk, src = measured_peaks()
            stages[-1]["tensor_roofline"] = {"bound": "tensor", "work_flops": work, "dag_ms": t_dag * 1e3,
                                             "achieved": work / t_dag / 1e12, "peak": pk, "unit": "TFLOP/s",
                                             "frac": work / t_dag / 1e12 / pk, "peak_source": "bf16 " + src}
        t_total += statistics.median(ms)
        todo = [todo[q] for q in range(len(todo)) if q not in set(ok)]
    D = geo.Batch([dict(pr, nb=nb, band=10 ** 6) for pr in probs], device=dev)
    dms, _, ddone = time_batch(geo, D, thetas, 3, dev)
    del D
    torch.cuda.empty_cache()
    ms_all, comp_all, nprob_all = gather_shards(
        {"ms": t_total, "completion_ms": completion[np.isfinite(completion)].tolist(), "problems": len(probs)}, world)
    good = np.array(comp_all)
    t_total = ms_all
    return {"ranks": world, "problems": nprob_all, "workload": "256 datasets, n ~ U[500, 8000] uniform locations, sigma2 ~ U[0.5, 2], beta ~ U[0.02, 0.3], "
                        "nu in {1/2, 1, 3/2}; one graph-captured evaluation = generation + one persistent launch "
                        "(factorization, forward solve, log-det and Eq. 2 of every problem)",
            "autotune_ms_by_tile": tune, "tile": nb, "band_stages": stages,
            "problems_by_band": {str(b if b < 10 ** 6 else "all FP64"): sum(1 for v in band_of.values() if v == b)
                                 for b in BATCH_BAND_LADDER},
            "unfactored": len(todo), "ms_per_batch": t_total,
            "per_problem_completion_p50_ms": float(np.percentile(good, 50)) if good.size else None,
            "per_problem_completion_p99_ms": float(np.percentile(good, 99)) if good.size else None,
            "evals_per_s": nall / (t_total / 1000.0), "tflops": flops / (t_total / 1000.0) / 1e12,
            "fp64_ms": statistics.median(dms), "fp64_evals_per_s": len(probs) / (statistics.median(dms) / 1000.0),
            "fp64_per_problem_completion_p50_ms": float(np.nanpercentile(ddone, 50)),
            "fp64_per_problem_completion_p99_ms": float(np.nanpercentile(ddone, 99)),
            "speedup_vs_fp64": statistics.median(dms) / t_total}


DST_BANDS = (1, 2, 4)
# far tier of the three-precision extension: (far_band, far_dist, products)
FAR_SWEEP = [(2, 0.0, 3), (4, 0.0, 3), (8, 0.0, 3), (16, 0.0, 3), (32, 0.0, 3), (8, 0.0, 1), (16, 0.0, 1),
             (32, 0.0, 1), (0, 0.2, 3), (0, 0.3, 3), (0, 0.5, 3), (0, 0.5, 1)]


def far_tile_count(x, y, nb, far_band, far_dist):
    """Off-band tiles of band 1 that the far rule marks (host count for the report)."""
    n = len(x)
    p = -(-n // nb)
    box = [(x[i * nb:(i + 1) * nb].min(), x[i * nb:(i + 1) * nb].max(), y[i * nb:(i + 1) * nb].min(),
            y[i * nb:(i + 1) * nb].max()) for i in range(p)]
    cnt = 0
    for j in range(p):
        for i in range(j + 1, p):
            f = far_band > 0 and i - j >= far_band
            if far_dist > 0:
                gx = max(0.0, box[j][0] - box[i][1], box[i][0] - box[j][1])
                gy = max(0.0, box[j][2] - box[i][3], box[i][2] - box[j][3])
                f = f or math.hypot(gx, gy) >= far_dist
            cnt += f
    return cnt, p * (p - 1) // 2
SERVE_SWEEP_RATES = (2.0, 5.0, 7.0, 10.0, 14.0, 20.0)
SERVE_SWEEP_WINDOW = 4.0
SERVE_DRAIN_S = 1.0   # a rate is sustained when the window's requests are all served within this after it


def run_serve(geo, dev, window):
    """Serving: 16 resident datasets (n ~ U[1k, 50k], four of them in [10k, 40k]
    hold a resident factor for kriging), Poisson arrivals at 200/s for `window`
    seconds, 70 % log-likelihood (random theta) and 30 % kriging (100 new
    points, nu 1/2 or 3/2), admission by an HBM budget of 120 GB; then the
    same mix at SERVE_SWEEP_RATES for SERVE_SWEEP_WINDOW seconds each, to
    locate the highest rate the server sustains."""
    import torch
    from paper_2003_05324_b300 import inputs, serve
    rng = np.random.default_rng(7)
    ns = [int(v) for v in rng.integers(1000, 50001, size=12)] + [int(v) for v in rng.integers(10000, 40001, size=4)]
    dss, truth = [], []
    for d, n in enumerate(ns):
        kr = d >= 12
        nu = float(rng.choice([0.5, 1.5])) if kr else 0.5
        # kriging data carry a measurement-error nugget (1e-4 sigma2): without
        # one the nu = 3/2 covariance of 10k-40k uniform points is numerically
        # singular for FP32 off-band storage
        th = geo.Theta(1.0, 0.1, nu, 1e-4 if kr else 0.0)
        x, y = inputs.uniform_points(n + (100 if kr else 0), seed=200 + d)
        z = (inputs.matern_field_rff(x, y, 1.0, 0.1, nu, seed=300 + d, nugget=1e-4) if kr
             else inputs.white_noise(n, seed=300 + d))
        xo, yo, zo = x[:n], y[:n], z[:n]
        perm = geo.morton_order(xo, yo)
        dss.append(dict(x=xo[perm], y=yo[perm], z=zo[perm], theta=th, nb=500, krige=kr))
        truth.append((x[n:], y[n:], z[n:]) if kr else None)
    S = serve.Server(dss, hbm_budget_bytes=120 << 30, nb=500)

    def arrivals(rate, win, rng):
        reqs, t, q = [], 0.0, 0
        while True:
            t += float(rng.exponential(1.0 / rate))
            if t > win:
                return reqs
            if rng.uniform() < 0.7:
                d = int(rng.integers(0, 16))
                reqs.append(serve.Request("loglik", d, theta=geo.Theta(float(rng.uniform(0.5, 2.0)),
                                                                        float(rng.uniform(0.02, 0.3)),
                                                                        dss[d]["theta"].nu, dss[d]["theta"].nugget),
                                          t_arrival=t, id=q))
            else:
                d = int(rng.integers(12, 16))
                xt, yt, _ = truth[d]
                reqs.append(serve.Request("krige", d, xnew=xt, ynew=yt, t_arrival=t, id=q))
            q += 1

    reqs = arrivals(200.0, window, rng)
    results, stats = S.run(reqs, admit_until=window)
    # arrival-rate sweep (same datasets and request mix, seed 8): every request
    # that arrives in the window is served (the queue drains after it); a rate
    # is sustained when the last of them completes within SERVE_DRAIN_S of the
    # end of the window -- above the knee the backlog, and with it the drain
    # time and the latency, grows with the window
    sweep = []
    rng_s = np.random.default_rng(8)
    for rate in SERVE_SWEEP_RATES:
        rq = arrivals(rate, SERVE_SWEEP_WINDOW, rng_s)
        b0 = S.batches
        _, st = S.run(rq)
        sweep.append({"rate_per_s": rate, "requests": len(rq), "completed": st["completed"],
                      "rejected": st["rejected"], "launches": S.batches - b0,
                      "drain_s": st["wall_s"] - SERVE_SWEEP_WINDOW,
                      "evals_per_s": st["evals_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"]})
    ok = [r["rate_per_s"] for r in sweep
          if r["completed"] + r["rejected"] == r["requests"] and r["drain_s"] <= SERVE_DRAIN_S]
    # kriging accuracy: MSPE of the served (mixed-precision) predictions and of
    # the FP64 path's, against the held-out field values
    mspe = []
    for d in range(12, 16):
        xt, yt, zt = truth[d]
        served = [r.value for r in results if r.kind == "krige" and r.dataset == d]
        if not served:
            continue
        ds = S.ds[d]
        ts = geo.TileStore(ds["n"], 500, 10 ** 6, geo.GEO_LP_SPLIT_BF16, device=dev)
        ts.matern(ds["x"], ds["y"], ds["theta"])
        ts.potrf()
        p64 = ts.krige(ds["x"], ds["y"], ds["z"], ds["theta"], torch.as_tensor(xt, device=dev),
                       torch.as_tensor(yt, device=dev)).cpu().numpy()
        m_mp, m_dp = float(np.mean((served[0] - zt) ** 2)), float(np.mean((p64 - zt) ** 2))
        mspe.append({"dataset_n": ds["n"], "mspe_mp": m_mp, "mspe_fp64": m_dp, "rel_diff": abs(m_mp - m_dp) / m_dp})
        del ts
    stats.update({"arrival_rate_per_s": 200, "window_s": window, "requests": len(reqs),
                  "datasets_n": ns, "hbm_budget_gb": 120, "kriging_mspe": mspe,
                  "rate_sweep": sweep, "sweep_window_s": SERVE_SWEEP_WINDOW, "sweep_drain_limit_s": SERVE_DRAIN_S,
                  "sustainable_rate_per_s": max(ok) if ok else None,
                  "note": "offered load exceeds capacity: requests still queued at the end are reported, not served"})
    return stats


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2003_05324_b300 import geo
    dev = torch.device("cuda", local)
    # CPU oracle baseline first (before heavy GPU work; rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(2)

    x, y, z = workload()
    perm = geo.morton_order(x, y)
    x, y, z = x[perm], y[perm], z[perm]
    n = len(z)
    th = geo.Theta(*THETA)
    X = torch.as_tensor(x, device=dev)
    Y = torch.as_tensor(y, device=dev)
    Z = torch.as_tensor(z, device=dev)
    lp = geo.GEO_LP_SPLIT_BF16 if args.lp == "bf16" else geo.GEO_LP_FP32
    ts = geo.TileStore(n, NB, args.band, lp, device=dev)
    gen_flags = (geo.GEO_FLAG_FP64_OFFBAND_GEN if args.gen64 else 0) | (geo.GEO_FLAG_FP64_DMMA if args.dmma else 0)
    ts.set_flags(gen_flags)
    stream = torch.cuda.current_stream(dev)
    flops = n ** 3 / 3.0

    res = torch.empty(3, dtype=torch.float64, device=dev)   # (log|Sigma|, Z' Sigma^-1 Z, l) on the device

    def eval_once(store):
        """One evaluation on the current stream: (seconds by CUDA events, l read from the device)."""
        out = torch.empty(3, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        store.loglik_async(X, Y, Z, th, out=out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        code, info = store.status()
        if code != 0:
            raise (geo.NotSPDError if code == geo.GEO_ERR_NOT_SPD else geo.GeoError)(code, "geo_loglik_async", info)
        return e0.elapsed_time(e1) / 1000.0, float(out[2])

    # warm-up (also the accuracy reference for this band)
    for _ in range(args.warmup):
        ts.loglik_async(X, Y, Z, th, out=res)
    torch.cuda.synchronize(dev)
    code, info = ts.status()
    if code != 0:
        raise SystemExit(f"device status {code} (info {info}) during warm-up")
    l_mp = float(res[2])

    # timed region: K steps back to back on the stream, CUDA events around them
    geo.profile_reset()
    geo.profile_enable(True)
    launches0 = geo.kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev0.record(stream)
    step_ev[0].record(stream)
    for s in range(args.steps):
        ts.loglik_async(X, Y, Z, th, out=res)
        step_ev[s + 1].record(stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    geo.profile_enable(False)
    launches = geo.kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1)
    step_ms = [step_ev[i].elapsed_time(step_ev[i + 1]) for i in range(args.steps)]
    ms = max_over_ranks(ms, world, dev)
    code, info = ts.status()
    if code != 0:
        raise SystemExit(f"device status {code} (info {info}) in the timed region")
    ms_step = ms / args.steps
    evals_per_s, tflops = replica_throughput(ms, world, args.steps, flops)

    # per-kernel live timings (CUDA events on each kernel's own stream)
    kern = {kind: geo.profile_read(kind) for kind in range(6)}
    rows, roofline = kernel_rows(ts, args, kern)
    gen = generation_row(ts, kern[5])
    if gen:
        rows.append(gen)

    # all-FP64 GPU paths: the accuracy reference and the throughput comparison.
    # The fastest one (FP64-accurate tensor-core updates) is the headline
    # comparator; the FP64-pipe (DMMA) path is reported beside it.
    fp64 = None
    if not args.no_fp64:
        ts64e = geo.TileStore(n, NB, 10 ** 6, geo.GEO_LP_SPLIT_BF16, device=dev)
        eval_once(ts64e)
        te, l64 = eval_once(ts64e)
        del ts64e
        fp64 = {"path": "all tiles FP64, FP64-accurate tensor-core updates (the fastest all-FP64 GPU path)",
                "seconds_per_eval": te, "tflops": flops / te / 1e12, "evals_per_s": 1.0 / te, "loglik": l64,
                "mp_speedup": te / (ms_step / 1000.0), "mp_rel_err": abs(l_mp - l64) / abs(l64)}
        if not args.no_dmma:
            ts64 = geo.TileStore(n, NB, 10 ** 6, geo.GEO_LP_FP32, device=dev)
            td, ld_ = eval_once(ts64)          # one evaluation (22 s): no separate warm-up
            del ts64
            fp64["fp64_pipe"] = {"path": "all tiles FP64, updates on the FP64 pipe (DMMA)",
                                 "seconds_per_eval": td, "tflops": flops / td / 1e12,
                                 "mp_speedup": td / (ms_step / 1000.0),
                                 "rel_diff_vs_tensor_fp64": abs(ld_ - l64) / abs(l64)}

    # end to end through the public blocking call, host buffers copied every step
    xh = torch.as_tensor(x).pin_memory()
    yh = torch.as_tensor(y).pin_memory()
    zh = torch.as_tensor(z).pin_memory()
    Xe, Ye, Ze = torch.empty_like(X), torch.empty_like(Y), torch.empty_like(Z)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Xe.copy_(xh, non_blocking=True)
        Ye.copy_(yh, non_blocking=True)
        Ze.copy_(zh, non_blocking=True)
        l_e2e = ts.loglik(Xe, Ye, Ze, th)[0]
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": flops / t_e2e / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 3 * 8 * n,
           "d2h_bytes_per_step": 3 * 8 + 3 * 4, "seconds_per_eval": t_e2e}

    # the band sweep of the configuration: bands 2, 4, 8 beside the timed band,
    # each with its error against the FP64 path
    sweep = None
    if not args.no_sweep:
        sweep = [{"band": ts.band, "seconds_per_eval": ms_step / 1000.0, "tflops": tflops, "loglik": l_mp}]
        for bb in (2, 4, 8):
            if bb == ts.band:
                continue
            tsb = geo.TileStore(n, NB, bb, lp, device=dev)
            tsb.set_flags(gen_flags)
            eval_once(tsb)
            tb, lb = eval_once(tsb)
            sweep.append({"band": bb, "seconds_per_eval": tb, "tflops": flops / tb / 1e12, "loglik": lb})
            del tsb
        for ent in sweep:
            if fp64:
                ent["rel_err_vs_fp64"] = abs(ent["loglik"] - fp64["loglik"]) / abs(fp64["loglik"])

    # the DST / IND approximation (Section V-B): tiles at distance >= d zeroed,
    # the kept ones FP64; NOT_SPD when the truncation is indefinite
    dst = []
    if not args.no_dst:
        for dd in DST_BANDS:
            tsd = geo.TileStore(n, NB, dd, geo.GEO_LP_SPLIT_BF16, device=dev)
            tsd.set_flags(geo.GEO_FLAG_DST)
            ent = {"d": dd}
            try:
                eval_once(tsd)
                td, ldst = eval_once(tsd)
                ent.update({"seconds_per_eval": td, "speedup_vs_mp": (ms_step / 1000.0) / td, "loglik": ldst})
                if fp64:
                    ent["rel_diff_vs_fp64"] = abs(ldst - fp64["loglik"]) / abs(fp64["loglik"])
            except geo.NotSPDError:
                ent["status"] = "not positive definite (the truncated covariance is indefinite)"
            dst.append(ent)
            del tsd

    # the far tier of the three-precision extension: error and time per rule
    far = []
    if not args.no_far and args.lp == "bf16" and ts.band == 1:
        for fb, fd, fp in FAR_SWEEP:
            tsf = geo.TileStore(n, NB, 1, geo.GEO_LP_SPLIT_BF16, device=dev)
            tsf.set_far(fb, X, Y, fd, fp)
            cnt, tot = far_tile_count(x, y, NB, fb, fd)
            ent = {"far_band": fb, "far_dist": fd, "products": fp, "far_tiles": cnt, "offband_tiles": tot}
            try:
                eval_once(tsf)
                tf, lf = eval_once(tsf)
                ent.update({"seconds_per_eval": tf, "tflops": flops / tf / 1e12, "loglik": lf,
                            "speedup_vs_mp": (ms_step / 1000.0) / tf})
                if fp64:
                    ent["rel_err_vs_fp64"] = abs(lf - fp64["loglik"]) / abs(fp64["loglik"])
                    ent["passes_1e-6_gate"] = ent["rel_err_vs_fp64"] <= 1e-6
            except geo.NotSPDError:
                ent["status"] = "not positive definite with this far tier"
            far.append(ent)
            del tsf

    # batched problems are independent: with several ranks each evaluates a
    # disjoint share (every rank takes part in the gather)
    batch = run_batch(geo, dev, rank, world) if not args.no_batch else None

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    p50 = statistics.median(step_ms)
    p99 = sorted(step_ms)[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)]
    out = {
        "metric": METRIC,
        "value": tflops, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32(fp16-slices)" if args.lp == "bf16" else "f64+f32",
        "data": "synthetic",
        "config": {"workload": f"loglik n={n} (200x200 jittered grid, Morton), Matern sigma2=1 beta=0.1 nu=0.5, "
                               f"tile {NB}, band {ts.band}, off-band "
                               f"{'FP16 slice products on the tensor cores' if args.lp == 'bf16' else 'FP32 FMA'}",
                   "n": n, "nb": NB, "band": ts.band,
                   "offband_products": "fp16-slices (8/12/12-bit, 6 tcgen05 products)" if args.lp == "bf16"
                   else "fp32-fma",
                   "offband_generation": "fp64-rounded" if args.gen64 else "compensated fp32",
                   "cache": "working set 3.3 GB of tiles >> 126 MB L2 (no flush needed)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "evals_per_s": evals_per_s, "p50_ms": p50, "p99_ms": p99,
        "loglik": l_mp, "loglik_e2e": l_e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": roofline,
        "tile_mix_roofline": tile_mix_roofline(rows, ts, ms_step),
        "kernels": rows,
        "fp64_path": fp64,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if sweep is not None:
        out["band_sweep"] = sweep
    if dst:
        out["dst"] = dst
    if far:
        out["far_tier_sweep"] = far
        ok = [e for e in far if e.get("passes_1e-6_gate")]
        out["far_tier_best"] = min(ok, key=lambda e: e["seconds_per_eval"]) if ok else None
    if batch is not None:
        out["batch"] = batch
    if not args.no_serve and world == 1:
        out["serving"] = run_serve(geo, dev, args.serve_window)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

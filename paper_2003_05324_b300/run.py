"""Evaluate the log-likelihood on the synthetic workload from the command line.

    python -m paper_2003_05324_b300.run --m 200 --nb 500 --band 1 --lp bf16 --reps 2

m x m jittered grid (seed 0) in Morton order, Matern sigma2 = 1, beta = 0.1,
nu = 0.5, measurements from the seeded spectral field simulation (seed 1) --
the same recipe as bench.py.  Prints l(theta), log|Sigma| and Z' Sigma^-1 Z and
the wall time of each repetition.  Used as the target of profiler captures.

--trace runs one more evaluation with the scheduler's task trace enabled
(geo_tiles_set_trace) and prints a summary of the records: per task type its
count, mean duration and summed time; the per-SM period of the off-band
tensor items and their copy / MMA / epilogue phases; tensor items finished
per 5 ms; the critical chain PC(k) of the last steps.  --trace-out FILE also
saves the raw records (numpy .npy).
"""
import argparse
import time

import numpy as np
import torch

from . import geo, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=200)
    ap.add_argument("--nb", type=int, default=500)
    ap.add_argument("--band", type=int, default=1)
    ap.add_argument("--lp", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--trace", action="store_true", help="trace one more evaluation and summarise it")
    ap.add_argument("--trace-out", default=None, help="save the raw trace records here (.npy)")
    a = ap.parse_args()
    x, y = inputs.jittered_grid(a.m, seed=0)
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=1)
    perm = geo.morton_order(x, y)
    x, y, z = x[perm], y[perm], z[perm]
    X, Y, Z = (torch.as_tensor(v, device="cuda") for v in (x, y, z))
    ts = geo.TileStore(len(z), a.nb, a.band, geo.GEO_LP_SPLIT_BF16 if a.lp == "bf16" else geo.GEO_LP_FP32)
    for r in range(a.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        l, ld, q = ts.loglik(X, Y, Z, geo.Theta(1.0, 0.1, 0.5))
        dt = time.perf_counter() - t0
        print(f"rep {r}: loglik {l:.12e} logdet {ld:.12e} quad {q:.12e}  {dt:.4f} s", flush=True)
    if a.trace:
        ts.enable_trace(8 << 20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        l, ld, q = ts.loglik(X, Y, Z, geo.Theta(1.0, 0.1, 0.5))
        print(f"traced: loglik {l:.12e}  {time.perf_counter() - t0:.4f} s", flush=True)
        recs = ts.read_trace()
        if a.trace_out:
            np.save(a.trace_out, recs)
        summarize_trace(recs)


def summarize_trace(r, out=print):
    """Summary of the task-trace records of one factorization (record types as
    in include/geo.h's geo_trace_rec)."""
    t0 = r["t_claim"][r["t_claim"] > 0].min()
    ms = lambda v: (v - t0) / 1e6
    span = ms(r["t_end"].max())
    out(f"records {len(r)}  span {span:.2f} ms")
    for ty in sorted(set(r["type"].tolist())):
        s = r[r["type"] == ty]
        d = (s["t_end"] - s["t_claim"]) / 1e3
        out(f"type {ty:2d}: n={len(s):8d}  duration us mean {d.mean():8.2f} p50 {np.median(d):8.2f}  sum {d.sum() / 1e3:9.1f} ms")
    off = r[r["type"] == 10]
    if len(off):
        per = np.concatenate([np.diff(np.sort(off[off["sm"] == sm]["t_ready"])) for sm in np.unique(off["sm"])]) / 1e3
        epi = (off["t_end"] - off["t_ready"]) / 1e3
        out("off-band item period per SM us: p10 %.2f p50 %.2f p90 %.2f | epilogue us p50 %.2f" %
            (*np.percentile(per, [10, 50, 90]), np.median(epi)))
    for ty, what, a, b in ((15, "MMA thread: wait for first stage", "t_claim", "t_ready"),
                           (15, "MMA thread: first stage to last MMA", "t_ready", "t_end"),
                           (16, "copy thread: take item to dependencies met", "t_claim", "t_ready"),
                           (16, "copy thread: dependencies to first copies", "t_ready", "t_end")):
        s = r[r["type"] == ty]
        if len(s):
            d = (s[b] - s[a]) / 1e3
            out(f"{what} us: p50 {np.median(d):.2f} mean {d.mean():.2f}")
    tc = r[(r["type"] == 10) | (r["type"] == 11)]
    if len(tc):
        h, _ = np.histogram(ms(tc["t_end"]), bins=np.arange(0, span + 5, 5))
        out("tensor items finished per 5 ms: " + " ".join(str(v) for v in h.tolist()))
    pc = r[r["type"] == 7]
    if len(pc):
        late = pc[pc["k"] >= pc["k"].max() * 0.55]
        out("PC(k), last 45 %% of steps: wait us %.1f, work us %.1f, steps %.3f ms apart" %
            (((late["t_ready"] - late["t_claim"]) / 1e3).mean(), ((late["t_end"] - late["t_ready"]) / 1e3).mean(),
             np.diff(np.sort(late["t_end"])).mean() / 1e6 if len(late) > 1 else float("nan")))
    for ty, what in ((12, "PC sub-step factor"), (13, "PC sub-step solve")):
        s = r[r["type"] == ty]
        if len(s):
            out(f"{what}: wait us {((s['t_ready'] - s['t_claim']) / 1e3).mean():.2f}, "
                f"work us {((s['t_end'] - s['t_ready']) / 1e3).mean():.2f}")


if __name__ == "__main__":
    main()

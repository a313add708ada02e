"""Evaluate the log-likelihood on the synthetic workload from the command line.

    python -m paper_2003_05324_b300.run --m 200 --nb 500 --band 1 --lp bf16 --reps 2

m x m jittered grid (seed 0) in Morton order, Matern sigma2 = 1, beta = 0.1,
nu = 0.5, measurements from the seeded spectral field simulation (seed 1) --
the same recipe as bench.py.  Prints l(theta), log|Sigma| and Z' Sigma^-1 Z and
the wall time of each repetition.  Used as the target of profiler captures.
"""
import argparse
import time

import torch

from . import geo, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=200)
    ap.add_argument("--nb", type=int, default=500)
    ap.add_argument("--band", type=int, default=1)
    ap.add_argument("--lp", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--reps", type=int, default=2)
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


if __name__ == "__main__":
    main()

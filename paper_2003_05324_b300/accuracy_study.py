"""Estimation and prediction accuracy of DP, MP and DST on synthetic data.

    python -m paper_2003_05324_b300.accuracy_study --m 100 --betas 0.03 0.1 0.3 --seeds 0 1

A reduced form of the paper's Monte-Carlo study (Section VIII-D): for each range
parameter theta2 (weak / medium / strong correlation) and seed,

* locations: an m x m jittered grid (seed), Morton order;
* measurements: an exact sample of the zero-mean Matern field with theta =
  (1, theta2, 1/2): Z = L w with L the all-FP64 GPU factor of Sigma(theta) and
  w standard normal (seed + 1000);
* a random 10 % of the points (seed + 2000) is held out for prediction;
* each method estimates theta on the rest with the library's Nelder-Mead MLE
  (same start, bounds and budget for all): DP (every tile FP64), MP with band
  1 and 2 (Algorithm 1), DST with d = 1 (independent blocks) and d = 2;
* with its estimate each method refactors and predicts the held-out values
  by simple kriging; the score is the mean square prediction error.

Prints one JSON line per (theta2, seed, method) and a summary table of the
estimates' distance to DP's and of the prediction errors.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import geo, inputs

METHODS = (("DP", 10 ** 6, 0), ("MP b=1", 1, 0), ("MP b=2", 2, 0), ("DST d=1", 1, geo.GEO_FLAG_DST),
           ("DST d=2", 2, geo.GEO_FLAG_DST))


def exact_field(x, y, theta, nb, seed, dev):
    """Z = L w: the all-FP64 factor of Sigma(theta) times standard normal w."""
    n = len(x)
    X, Y = (torch.as_tensor(v, device=dev) for v in (x, y))
    ts = geo.TileStore(n, nb, 10 ** 6, geo.GEO_LP_SPLIT_BF16, device=dev)
    ts.matern(X, Y, theta)
    ts.potrf()
    L = ts.to_dense()
    w = torch.as_tensor(inputs.white_noise(n, seed=seed), device=dev)
    z = (L @ w).cpu().numpy()
    del L, ts
    torch.cuda.empty_cache()
    return z


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=100)
    ap.add_argument("--nb", type=int, default=500)
    ap.add_argument("--betas", type=float, nargs="+", default=[0.03, 0.1, 0.3])
    ap.add_argument("--seeds", type=int, nargs="+", default=[0, 1])
    ap.add_argument("--evals", type=int, default=200)
    ap.add_argument("--holdout", type=float, default=0.1)
    a = ap.parse_args()
    dev = torch.device("cuda")
    rows = []
    for beta in a.betas:
        for seed in a.seeds:
            x, y = inputs.jittered_grid(a.m, seed=seed)
            perm = geo.morton_order(x, y)
            x, y = x[perm], y[perm]
            th_true = geo.Theta(1.0, beta, 0.5)
            z = exact_field(x, y, th_true, a.nb, seed + 1000, dev)
            n = len(z)
            test = np.zeros(n, dtype=bool)
            test[np.random.default_rng(seed + 2000).choice(n, int(round(a.holdout * n)), replace=False)] = True
            tr, te = ~test, test        # the training points keep their Morton order
            Xtr, Ytr, Ztr = (torch.as_tensor(np.ascontiguousarray(v[tr]), device=dev) for v in (x, y, z))
            Xte, Yte = (torch.as_tensor(np.ascontiguousarray(v[te]), device=dev) for v in (x, y))
            zte = z[te]
            ntr = int(tr.sum())
            for name, band, flags in METHODS:
                ts = geo.TileStore(ntr, a.nb, band, geo.GEO_LP_SPLIT_BF16, device=dev)
                if flags:
                    ts.set_flags(flags)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                try:
                    r = ts.mle(Xtr, Ytr, Ztr, geo.Theta(0.5, 0.05, 0.4), max_evals=a.evals)
                except geo.NotSPDError:   # the truncated covariance is indefinite at the start
                    row = {"theta2": beta, "seed": seed, "method": name, "n_train": ntr,
                           "status": "not positive definite at the starting theta: no estimate"}
                    rows.append(row)
                    print(json.dumps(row), flush=True)
                    continue
                secs = time.perf_counter() - t0
                th = r["theta"]
                row = {"theta2": beta, "seed": seed, "method": name, "n_train": ntr, "n_test": int(te.sum()),
                       "theta_hat": [th.sigma2, th.beta, th.nu], "loglik": r["loglik"], "evals": r["evals"],
                       "not_spd_evals": r["not_spd"], "seconds": secs}
                try:
                    ts.matern(Xtr, Ytr, th)
                    ts.potrf()
                    zhat = ts.krige(Xtr, Ytr, Ztr, th, Xte, Yte).cpu().numpy()
                    row["mspe"] = float(np.mean((zhat - zte) ** 2))
                except geo.NotSPDError:
                    row["mspe"] = None      # no positive definite factor at the estimate
                rows.append(row)
                print(json.dumps(row), flush=True)
                del ts
                torch.cuda.empty_cache()
    # summary: distance of each estimate to DP's on the same data, prediction error
    print("\n| theta2 | method | max rel. distance of theta-hat to DP's (over seeds) | mean MSPE | MSPE / DP's |")
    print("|---|---|---|---|---|")
    for beta in a.betas:
        dp = {r["seed"]: r for r in rows if r["theta2"] == beta and r["method"] == "DP"}
        for name, _, _ in METHODS:
            rs = [r for r in rows if r["theta2"] == beta and r["method"] == name and "theta_hat" in r]
            if not rs:
                print(f"| {beta} | {name} | no estimate (indefinite) | - | - |")
                continue
            dist = max(max(abs(u - v) / abs(v) for u, v in zip(r["theta_hat"], dp[r["seed"]]["theta_hat"]))
                       for r in rs)
            ms = [r["mspe"] for r in rs if r["mspe"] is not None]
            rel = [r["mspe"] / dp[r["seed"]]["mspe"] for r in rs if r["mspe"] is not None]
            print(f"| {beta} | {name} | {dist:.2e} | {np.mean(ms) if ms else float('nan'):.4e} | "
                  f"{np.mean(rel) if rel else float('nan'):.4f} |")


if __name__ == "__main__":
    main()

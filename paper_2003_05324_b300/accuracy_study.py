"""Estimation and prediction accuracy of DP, MP and DST on synthetic data.

    python -m paper_2003_05324_b300.accuracy_study --m 200 --betas 0.03 0.1 0.3 --seeds 0 1 2 \
        --out study.jsonl

A reduced form of the paper's Monte-Carlo study (Section VIII-D): for each range
parameter theta2 (weak / medium / strong correlation) and seed,

* locations: an m x m jittered grid (seed), Morton order (m = 200: the
  paper's 40K points);
* measurements: an exact sample of the zero-mean Matern field with theta =
  (1, theta2, 1/2): Z = L w with L the all-FP64 GPU factor of Sigma(theta) and
  w standard normal (seed + 1000);
* each method estimates theta on all points with the library's Nelder-Mead
  MLE (same start, bounds and budget for all): DP (every tile FP64), MP with
  band 1 (Algorithm 1) and DST with d = 1 (independent blocks); the number of
  likelihood evaluations and simplex iterations each needed is recorded;
* prediction by 10-fold cross-validation: the points are split into 10 random
  folds (seed + 2000); each fold is predicted by simple kriging from the other
  nine with the method's own estimate and arithmetic; the score is the mean
  square prediction error over all points.

Every row is printed as one JSON line (and appended to --out), followed by a
summary table: the largest relative distance of each method's estimate to
DP's, the mean MSPE and its ratio to DP's, and the evaluations per estimate.
With --resume the rows already in --out are kept and only the missing
(theta2, seed, method) rows are computed; the summary covers all of them.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import geo, inputs

METHODS = {"DP": (10 ** 6, 0), "MP b=1": (1, 0), "MP b=2": (2, 0), "DST d=1": (1, geo.GEO_FLAG_DST),
           "DST d=2": (2, geo.GEO_FLAG_DST)}


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


def cv_mspe(x, y, z, theta, nb, band, flags, folds, seed, dev):
    """10-fold cross-validated MSPE: each fold kriged from the others with the
    given arithmetic (None when a factor is not positive definite)."""
    n = len(z)
    fold = np.random.default_rng(seed).permutation(n) % folds
    se = 0.0
    for f in range(folds):
        tr, te = fold != f, fold == f      # the training points keep their Morton order
        X, Y, Z = (torch.as_tensor(np.ascontiguousarray(v[tr]), device=dev) for v in (x, y, z))
        Xn, Yn = (torch.as_tensor(np.ascontiguousarray(v[te]), device=dev) for v in (x, y))
        ts = geo.TileStore(int(tr.sum()), nb, band, geo.GEO_LP_SPLIT_BF16, device=dev)
        if flags:
            ts.set_flags(flags)
        try:
            ts.matern(X, Y, theta)
            ts.potrf()
        except geo.NotSPDError:
            return None
        zhat = ts.krige(X, Y, Z, theta, Xn, Yn).cpu().numpy()
        se += float(np.sum((zhat - z[te]) ** 2))
        del ts
    return se / n


def run_study(m, nb, betas, seeds, evals, methods, folds=10, dev=None, emit=print, done=()):
    """The rows of every (theta2, seed, method) not in `done` (rows of an
    earlier run, returned with the new ones)."""
    dev = dev or torch.device("cuda")
    rows = list(done)
    have = {(r["theta2"], r["seed"], r["method"]) for r in rows}
    for beta in betas:
        for seed in seeds:
            todo = [name for name in methods if (beta, seed, name) not in have]
            if not todo:
                continue
            x, y = inputs.jittered_grid(m, seed=seed)
            perm = geo.morton_order(x, y)
            x, y = x[perm], y[perm]
            th_true = geo.Theta(1.0, beta, 0.5)
            z = exact_field(x, y, th_true, nb, seed + 1000, dev)
            n = len(z)
            X, Y, Z = (torch.as_tensor(v, device=dev) for v in (x, y, z))
            for name in todo:
                band, flags = METHODS[name]
                ts = geo.TileStore(n, nb, band, geo.GEO_LP_SPLIT_BF16, device=dev)
                if flags:
                    ts.set_flags(flags)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                try:
                    r = ts.mle(X, Y, Z, geo.Theta(0.5, 0.05, 0.4), max_evals=evals)
                except geo.NotSPDError:   # the truncated covariance is indefinite at the start
                    row = {"theta2": beta, "seed": seed, "method": name, "n": n,
                           "status": "not positive definite at the starting theta: no estimate"}
                    rows.append(row)
                    emit(json.dumps(row))
                    continue
                secs = time.perf_counter() - t0
                del ts
                torch.cuda.empty_cache()
                th = r["theta"]
                row = {"theta2": beta, "seed": seed, "method": name, "n": n,
                       "theta_hat": [th.sigma2, th.beta, th.nu], "loglik": r["loglik"], "evals": r["evals"],
                       "iterations": r["iterations"], "not_spd_evals": r["not_spd"], "seconds": secs,
                       "cv_folds": folds}
                t0 = time.perf_counter()
                row["mspe"] = cv_mspe(x, y, z, th, nb, band, flags, folds, seed + 2000, dev)
                row["cv_seconds"] = time.perf_counter() - t0
                rows.append(row)
                emit(json.dumps(row))
    return rows


def summary(rows, betas, methods):
    """Per theta2 and method: the largest relative distance of the estimate to
    DP's on the same data, the mean CV MSPE and its mean ratio to DP's, and the
    mean evaluations / iterations of the estimator."""
    out = []
    for beta in betas:
        dp = {r["seed"]: r for r in rows if r["theta2"] == beta and r["method"] == "DP" and "theta_hat" in r}
        for name in methods:
            rs = [r for r in rows if r["theta2"] == beta and r["method"] == name and "theta_hat" in r]
            if not rs:
                out.append({"theta2": beta, "method": name, "status": "no estimate (indefinite)"})
                continue
            dist = [max(abs(u - v) / abs(v) for u, v in zip(r["theta_hat"], dp[r["seed"]]["theta_hat"]))
                    for r in rs if r["seed"] in dp]
            ms = [r["mspe"] for r in rs if r["mspe"] is not None]
            rel = [r["mspe"] / dp[r["seed"]]["mspe"] for r in rs
                   if r["mspe"] is not None and r["seed"] in dp and dp[r["seed"]]["mspe"]]
            out.append({"theta2": beta, "method": name, "datasets": len(rs),
                        "max_rel_dist_to_dp": max(dist) if dist else None,
                        "median_rel_dist_to_dp": float(np.median(dist)) if dist else None,
                        "mean_mspe": float(np.mean(ms)) if ms else None,
                        "mean_mspe_ratio_to_dp": float(np.mean(rel)) if rel else None,
                        "mean_evals": float(np.mean([r["evals"] for r in rs])),
                        "mean_iterations": float(np.mean([r["iterations"] for r in rs])),
                        "mean_seconds": float(np.mean([r["seconds"] for r in rs]))})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=200)
    ap.add_argument("--nb", type=int, default=500)
    ap.add_argument("--betas", type=float, nargs="+", default=[0.03, 0.1, 0.3])
    ap.add_argument("--seeds", type=int, nargs="+", default=[0, 1, 2])
    ap.add_argument("--evals", type=int, default=150)
    ap.add_argument("--folds", type=int, default=10)
    ap.add_argument("--methods", nargs="+", default=["DP", "MP b=1", "DST d=1"], choices=list(METHODS))
    ap.add_argument("--out", default=None, help="append every JSON line to this file")
    ap.add_argument("--resume", action="store_true", help="keep the rows already in --out, compute the rest")
    a = ap.parse_args()
    done = []
    if a.resume and a.out:
        try:
            with open(a.out) as fh:
                done = [r for r in map(json.loads, filter(str.strip, fh)) if "method" in r and "summary" not in r]
        except FileNotFoundError:
            pass

    def emit(line):
        print(line, flush=True)
        if a.out:
            with open(a.out, "a") as fh:
                fh.write(line + "\n")

    rows = run_study(a.m, a.nb, a.betas, a.seeds, a.evals, a.methods, a.folds, emit=emit, done=done)
    for s in summary(rows, a.betas, a.methods):
        emit(json.dumps({"summary": s}))


if __name__ == "__main__":
    main()

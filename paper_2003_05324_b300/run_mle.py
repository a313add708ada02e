"""Maximum likelihood estimation on a synthetic dataset from the command line.

    python -m paper_2003_05324_b300.run_mle --m 360 --nb 720 --band 3 --nu 1.0 \
        --beta 0.03 --nugget 1e-8 --evals 60 --fp64-mle

m x m jittered grid (seed 0) in Morton order; measurements simulated from the
Matern field with the given (sigma2, beta, nu) and nugget by random Fourier
features (seed 1); the Nelder-Mead estimator (geo_mle) from
theta0 = (0.5, 0.05, 0.5) with the given evaluation budget.  Prints one JSON
line per estimate as soon as it is done: theta-hat, l(theta-hat), evaluations,
wall time per evaluation, and the arithmetic (band, tile, in-band updates on
the tensor cores or the FP64 pipe).

--fp64-mle then runs the same estimator, same start and budget, with every tile
FP64 (the all-FP64 GPU path, FP64-accurate tensor-core updates) and prints the
relative distance of the mixed-precision theta-hat to it, parameter by
parameter (Section IV-C's comparison of the two estimates at a matched
evaluation budget).  --out appends every JSON line to a file.

--journal-dir DIR runs each estimate in chunks of --chunk evaluations and
keeps geo_mle's evaluation journal in DIR after every chunk: a run that is
stopped resumes from the journal (the journaled evaluations are replayed, not
recomputed) and gives the same estimate as an uninterrupted one.

--mp-record FILE takes the mixed-precision estimate from a JSON line that an
earlier run wrote (the first line of FILE whose "estimate" is "mixed
precision" and whose n, nb and band match) instead of running it again, so
the all-FP64 estimate can run on its own.
"""
import argparse
import json
import os
import time

import numpy as np
import torch

from . import geo, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=360)
    ap.add_argument("--nb", type=int, default=720)
    ap.add_argument("--band", type=int, default=3)
    ap.add_argument("--sigma2", type=float, default=1.0)
    ap.add_argument("--beta", type=float, default=0.03)
    ap.add_argument("--nu", type=float, default=1.0)
    ap.add_argument("--nugget", type=float, default=1e-8)
    ap.add_argument("--evals", type=int, default=60)
    ap.add_argument("--profile", action="store_true", help="Eq. 3: sigma2 profiled")
    ap.add_argument("--dmma", action="store_true")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="after the estimate, evaluate l at theta-hat and theta-true with every tile FP64")
    ap.add_argument("--fp64-mle", action="store_true",
                    help="also run the estimator with every tile FP64 and compare the two estimates")
    ap.add_argument("--out", default=None, help="append the JSON lines to this file")
    ap.add_argument("--journal-dir", default=None, help="keep resumable evaluation journals here")
    ap.add_argument("--chunk", type=int, default=10, help="evaluations per chunk with --journal-dir")
    ap.add_argument("--mp-record", default=None, help="take the mixed-precision estimate from this JSON-lines file")
    a = ap.parse_args()

    def emit(rec):
        line = json.dumps(rec)
        print(line, flush=True)
        if a.out:
            with open(a.out, "a") as fh:
                fh.write(line + "\n")

    x, y = inputs.jittered_grid(a.m, seed=0)
    perm = geo.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, a.sigma2, a.beta, a.nu, seed=1, nugget=a.nugget)
    X, Y, Z = (torch.as_tensor(v, device="cuda") for v in (x, y, z))
    n = len(z)
    th0 = geo.Theta(0.5, 0.05, 0.5, a.nugget)
    th_true = geo.Theta(a.sigma2, a.beta, a.nu, a.nugget)

    def estimate(band, label):
        ts = geo.TileStore(n, a.nb, band, geo.GEO_LP_SPLIT_BF16)
        if a.dmma:
            ts.set_flags(geo.GEO_FLAG_FP64_DMMA)
        journal, jpath = None, None
        if a.journal_dir:
            os.makedirs(a.journal_dir, exist_ok=True)
            jpath = os.path.join(a.journal_dir, "mle_journal_band%d%s.json" % (ts.band, "_profile" if a.profile else ""))
            journal = {"records": np.zeros((a.evals, 4)), "len": 0}
            if os.path.exists(jpath):
                saved = json.load(open(jpath))
                journal["records"][:len(saved)] = np.array(saved, dtype=np.float64).reshape(-1, 4)
                journal["len"] = len(saved)
        done0 = journal["len"] if journal else 0
        l_true, t_eval = None, None
        if done0 == 0:   # (a resumed run skips this extra evaluation)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            l_true = ts.loglik(X, Y, Z, th_true)[0]
            t_eval = time.perf_counter() - t0
        t0 = time.perf_counter()
        if journal is None:
            r = ts.mle(X, Y, Z, th0, max_evals=a.evals, profile=a.profile)
        else:
            budget = done0
            while True:
                budget = min(a.evals, budget + a.chunk)
                r = ts.mle(X, Y, Z, th0, max_evals=budget, profile=a.profile, journal=journal)
                json.dump(journal["records"][:journal["len"]].tolist(), open(jpath, "w"))
                if budget >= a.evals or r["evals"] < budget:   # budget spent, or converged earlier
                    break
        wall = time.perf_counter() - t0
        new_evals = max(r["evals"] - done0, 1)
        th = r["theta"]
        rec = {"estimate": label, "n": n, "nb": a.nb, "band": ts.band, "seconds_first_eval": t_eval,
               "loglik_theta_true": l_true, "theta_true": [a.sigma2, a.beta, a.nu, a.nugget],
               "theta_hat": [th.sigma2, th.beta, th.nu], "loglik": r["loglik"], "evals": r["evals"],
               "iterations": r["iterations"], "not_spd": r["not_spd"], "seconds": wall,
               "evals_replayed_from_journal": done0,
               "seconds_per_eval": wall / new_evals,
               "tflops_per_eval": n ** 3 / 3.0 / (wall / new_evals) / 1e12, "profile": a.profile,
               "inband_updates": "fp64 pipe" if a.dmma else "tensor cores (FP64-accurate)"}
        return ts, rec

    if a.mp_record:
        mp, ts = None, None
        for line in open(a.mp_record):
            rec = json.loads(line)
            if rec.get("estimate") == "mixed precision" and (rec["n"], rec["nb"], rec["band"]) == (n, a.nb, a.band):
                mp = rec
                break
        if mp is None:
            raise SystemExit("no mixed-precision estimate for n=%d nb=%d band=%d in %s" % (n, a.nb, a.band, a.mp_record))
        if a.compare_fp64:
            raise SystemExit("--compare-fp64 needs the mixed-precision store: run without --mp-record")
    else:
        ts, mp = estimate(a.band, "mixed precision")
        emit(mp)
    th = mp["theta_hat"]
    if a.compare_fp64:
        l_mp_hat = mp["loglik"]
        del ts
        torch.cuda.empty_cache()
        t64 = geo.TileStore(n, a.nb, 10 ** 6, geo.GEO_LP_SPLIT_BF16)
        t0 = time.perf_counter()
        l64_true = t64.loglik(X, Y, Z, th_true)[0]
        sec64 = time.perf_counter() - t0
        l64_hat = t64.loglik(X, Y, Z, geo.Theta(th[0], th[1], th[2], a.nugget))[0]
        emit({"compare": "FP64 likelihood at the mixed-precision estimate", "seconds_fp64_eval": sec64,
              "loglik_fp64_theta_true": l64_true, "loglik_fp64_theta_hat": l64_hat,
              "rel_err_theta_true": (abs(mp["loglik_theta_true"] - l64_true) / abs(l64_true)
                                     if mp["loglik_theta_true"] is not None else None),
              "rel_err_theta_hat": abs(l_mp_hat - l64_hat) / abs(l64_hat)})
        del t64
    else:
        del ts
    torch.cuda.empty_cache()
    if a.fp64_mle:
        t64, dp = estimate(10 ** 6, "all tiles FP64")
        emit(dp)
        names = ("sigma2", "beta", "nu")
        emit({"compare": "mixed-precision theta-hat against the all-FP64 theta-hat (same start and budget)",
              "rel_err": {nm: abs(th[q] - dp["theta_hat"][q]) / abs(dp["theta_hat"][q]) for q, nm in enumerate(names)},
              "max_rel_err": max(abs(th[q] - dp["theta_hat"][q]) / abs(dp["theta_hat"][q]) for q in range(3)),
              "same_path": mp["evals"] == dp["evals"] and mp["iterations"] == dp["iterations"],
              "mp_speedup_per_eval": dp["seconds_per_eval"] / mp["seconds_per_eval"]})


if __name__ == "__main__":
    main()

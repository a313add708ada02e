"""Write the oracle's own mixed-precision MLE deviation (oracle calls only).

mle_alg1.json: for each dataset of the mixed-precision MLE test (jittered
m x m grid with the given seed, Morton order, measurements from the seeded
spectral field with seed + 1; theta_true = (1, 0.1, 1/2)), the estimate
theta-hat maximising Eq. 2 (or Eq. 3 with profile) with the dense FP64
likelihood, and with the likelihood of the oracle's Algorithm 1 factor
(tile nb, diag_thick 1: FP32 storage and FP32 BLAS beyond the diagonal), both
by the oracle's Nelder-Mead from theta0 = (0.5, 0.05, 0.5) run to convergence
(500 evaluations at most, xtol 1e-7), and the relative deviation of each
parameter (Section IV-C: the estimate of the mixed-precision method against
the double-precision one).

Run: python tests/golden/make_mle_alg1.py [--workers 8]
(hours on 8 cores: the n = 6,400 cases need ~30 s per Algorithm 1 evaluation)
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

# (m, nb, profile, seeds): the datasets of the GPU mixed-precision MLE test
CASES = [(40, 200, False, (5, 6, 7, 8, 9)), (40, 200, True, (5, 6, 7, 8, 9)), (80, 400, False, (5, 6, 7))]
THETA0 = (0.5, 0.05, 0.5)
KW = dict(max_evals=500, xtol=1e-7)


def _one(job):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    from oracle import geo_oracle as O
    from paper_2003_05324_b300 import inputs
    m, nb, profile, seed, kind = job
    x, y = inputs.jittered_grid(m, seed=seed)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=seed + 1)
    evaluate = None
    if kind == "alg1":
        def evaluate(th):
            L, info = O.mp_tile_cholesky(O.covariance(x, y, theta=th), nb, 1)
            return None if info != 0 else O.factor_logdet_quad(L, z)
    t0 = time.time()
    r = O.mle(x, y, z, O.Theta(*THETA0), profile=profile, evaluate=evaluate, **KW)
    th = r["theta"]
    return job, dict(theta=[th.sigma2, th.beta, th.nu], loglik=r["loglik"], evals=r["evals"],
                     iterations=r["iterations"], seconds=time.time() - t0)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--out", default=os.path.join(HERE, "mle_alg1.json"))
    a = ap.parse_args()
    jobs = [(m, nb, prof, s, kind) for (m, nb, prof, seeds) in CASES for s in seeds for kind in ("fp64", "alg1")]
    jobs.sort(key=lambda j: -j[0])   # the long n = 6,400 runs first
    res = {}
    with mp.get_context("spawn").Pool(a.workers) as pool:
        for job, r in pool.imap_unordered(_one, jobs):
            res[job] = r
            print(job, r, flush=True)
    out = {"theta0": list(THETA0), "max_evals": KW["max_evals"], "xtol": KW["xtol"], "band": 1, "cases": []}
    for (m, nb, prof, seeds) in CASES:
        for s in seeds:
            dp, al = res[(m, nb, prof, s, "fp64")], res[(m, nb, prof, s, "alg1")]
            dev = [abs(a - b) / abs(b) for a, b in zip(al["theta"], dp["theta"])]
            out["cases"].append({"m": m, "n": m * m, "nb": nb, "profile": prof, "seed": s, "fp64": dp,
                                 "alg1": al, "rel_dev": dev})
    with open(a.out, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", a.out)


if __name__ == "__main__":
    main()

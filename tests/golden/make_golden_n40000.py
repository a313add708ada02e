"""Write golden log-likelihood values at n = 40,000, computed by the oracle only.

loglik_n40000.json: the benchmark's workload -- n = 40,000 (200 x 200 jittered
grid, seed 0, Morton order), Matern sigma2 = 1, beta = 0.1, nu = 0.5, no
nugget, measurements from the seeded spectral field simulation (seed 1) --
with the FP64 log-likelihood of Eq. 2 and the oracle's Algorithm 1 value for
tile 500 and band 1.

At this size two things differ from the smaller golden script:

* the oracle's one-shot `covariance` would hold four dense n x n arrays at
  once, so the matrix is assembled from row blocks of the oracle's
  cross-covariance (with no nugget the diagonal entries are C(0) = sigma2
  either way);
* the host LAPACK's dense dpotrf ends in a segmentation fault on a 40,000 x
  40,000 matrix, so the FP64 factor is the oracle's tile Cholesky with every
  tile FP64 (Algorithm 1 with band >= p: 500 x 500 LAPACK calls only), which
  the CPU tests pin to the dense factor.

Each value runs in its own process so that at most ~45 GB is held:

    python tests/golden/make_golden_n40000.py          # both, then merge (~30 min on 8 cores)
    python tests/golden/make_golden_n40000.py fp64     # one part, printed as JSON
    python tests/golden/make_golden_n40000.py mp
"""
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import geo_oracle as O  # noqa: E402
from paper_2003_05324_b300 import inputs  # noqa: E402

M, NB, BAND = 200, 500, 1
THETA = (1.0, 0.1, 0.5, 0.0)


def workload():
    x, y = inputs.jittered_grid(M, seed=0)
    z = inputs.matern_field_rff(x, y, THETA[0], THETA[1], THETA[2], seed=1)
    perm = O.morton_order(x, y)
    return x[perm], y[perm], z[perm]


def covariance_blocked(x, y, th, rows=2000):
    n = len(x)
    S = np.empty((n, n), dtype=np.float64)
    for r0 in range(0, n, rows):
        S[r0:r0 + rows] = O.covariance(x[r0:r0 + rows], y[r0:r0 + rows], x, y, theta=th)
    return S


def part(which):
    x, y, z = workload()
    n = len(z)
    th = O.Theta(*THETA)
    t0 = time.time()
    S = covariance_blocked(x, y, th)
    L, info = O.mp_tile_cholesky(S, NB, 10 ** 6 if which == "fp64" else BAND)
    assert info == 0, info
    del S
    ld, q = O.factor_logdet_quad(L, z)
    return {"loglik": -0.5 * n * math.log(2 * math.pi) - 0.5 * ld - 0.5 * q, "logdet": ld, "quad": q,
            "seconds": time.time() - t0}


def main():
    if len(sys.argv) > 1:
        print(json.dumps(part(sys.argv[1])), flush=True)
        return
    res = {}
    for which in ("fp64", "mp"):
        out = subprocess.run([sys.executable, os.path.abspath(__file__), which], capture_output=True, text=True,
                             check=True).stdout
        res[which] = json.loads(out.strip().splitlines()[-1])
    n = M * M
    fp64, mp = res["fp64"], res["mp"]
    doc = {"n": n, "nb": NB, "theta": list(THETA), "grid": "200x200 jittered, seed 0, Morton",
           "z": "matern_field_rff(sigma2=1, beta=0.1, nu=0.5, seed=1), permuted with the points",
           "fp64": {k: fp64[k] for k in ("loglik", "logdet", "quad")},
           "mp": {str(BAND): {k: mp[k] for k in ("loglik", "logdet", "quad")}},
           "mp_rel_err": {str(BAND): abs(mp["loglik"] - fp64["loglik"]) / abs(fp64["loglik"])},
           "seconds": {"fp64": fp64["seconds"], "mp": mp["seconds"]}}
    with open(os.path.join(HERE, "loglik_n40000.json"), "w") as fh:
        json.dump(doc, fh, indent=1)
    print(json.dumps(doc))


if __name__ == "__main__":
    main()

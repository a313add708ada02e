"""Write golden log-likelihood values computed by the oracle only.

loglik_n22500.json: n = 22,500 (150 x 150 jittered grid, seed 0, Morton order),
Matern sigma2 = 1, beta = 0.1, nu = 0.5, measurements from the seeded spectral
field simulation (seed 1): the FP64 log-likelihood of Eq. 2 (dense Cholesky)
and the oracle's Algorithm 1 value for tile 500 and bands 1, 2, 4.

Run: python tests/golden/make_golden.py   (a few minutes on 8 cores, ~20 GB RAM)
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import geo_oracle as O  # noqa: E402
from paper_2003_05324_b300 import inputs  # noqa: E402


def main():
    m, nb = 150, 500
    x, y = inputs.jittered_grid(m, seed=0)
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=1)
    perm = O.morton_order(x, y)
    x, y, z = x[perm], y[perm], z[perm]
    n = len(z)
    th = O.Theta(1.0, 0.1, 0.5)
    t0 = time.time()
    S = O.covariance(x, y, theta=th)
    L, info = O.dense_factor(S)
    assert info == 0
    ld, q = O.factor_logdet_quad(L, z)
    del L
    out = {"n": n, "nb": nb, "theta": [1.0, 0.1, 0.5, 0.0], "grid": "150x150 jittered, seed 0, Morton",
           "z": "matern_field_rff(sigma2=1, beta=0.1, nu=0.5, seed=1), permuted with the points",
           "fp64": {"loglik": -0.5 * n * math.log(2 * math.pi) - 0.5 * ld - 0.5 * q, "logdet": ld, "quad": q},
           "mp": {}}
    for band in (1, 2, 4):
        Lm, info = O.mp_tile_cholesky(S, nb, band)
        assert info == 0
        ldm, qm = O.factor_logdet_quad(Lm, z)
        del Lm
        out["mp"][str(band)] = {"loglik": -0.5 * n * math.log(2 * math.pi) - 0.5 * ldm - 0.5 * qm,
                                "logdet": ldm, "quad": qm}
    out["seconds"] = time.time() - t0
    with open(os.path.join(HERE, "loglik_n22500.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

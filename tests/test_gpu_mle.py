"""Maximum likelihood estimation on the GPU (geo_mle, Section IV-C).

* The FP64 GPU path follows the oracle's simplex step for step: with the same
  theta0 and budget, the two objectives agree to ~1e-13, so the evaluation and
  iteration counts are equal and theta-hat agrees to 1e-9 (full and profiled
  likelihood; FP64 pipe and tensor-core FP64 updates).
* The mixed-precision estimate against the FP64 estimate, both run to
  convergence, dataset by dataset against the oracle's own Algorithm 1
  (tests/golden/mle_alg1.json, oracle calls only).  The FP32 storage of the
  off-band tiles leaves the likelihood surface with rounding noise that moves
  the optimum along the sigma2-beta ridge: the oracle's Algorithm 1 moves it by
  up to 2.3e-3 on single datasets at n = 1,600 (median 8e-4) and by up to 5e-3
  at n = 6,400 (median 2.2e-3).  So each dataset's GPU deviation must stay
  within three times the oracle's deviation on the same dataset (plus 1e-3),
  and the median over datasets within the stated 1e-3 gate at n = 1,600 and
  within twice the oracle's median at n = 6,400.
* 1D Markov data: the FP64 GPU estimate equals the closed-form argmax.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import geo_oracle as O  # noqa: E402
from paper_2003_05324_b300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_05324_b300 import geo
    return geo


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def grid_problem(m, seed, th):
    x, y = inputs.jittered_grid(m, seed=seed)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, th[0], th[1], th[2], seed=seed + 1)
    return x, y, z


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("profile", [False, True])
@pytest.mark.parametrize("updates", ["fp64-pipe", "tensor"])
def test_fp64_mle_follows_the_oracle(G, profile, updates):
    x, y, z = grid_problem(20, 3, (1.0, 0.1, 0.5))       # n = 400
    th0 = (0.5, 0.05, 0.5)
    want = O.mle(x, y, z, O.Theta(*th0), max_evals=60, profile=profile)
    mode = G.GEO_LP_FP32 if updates == "fp64-pipe" else G.GEO_LP_SPLIT_BF16
    ts = G.TileStore(400, 96, 10, mode)                    # band >= p: all tiles FP64
    got = ts.mle(dev(x), dev(y), dev(z), G.Theta(*th0), max_evals=60, profile=profile)
    assert got["evals"] == want["evals"] and got["iterations"] == want["iterations"]
    for a in ("sigma2", "beta", "nu"):
        assert rel(getattr(got["theta"], a), getattr(want["theta"], a)) <= 1e-9, a
    assert rel(got["loglik"], want["loglik"]) <= 1e-11


def _golden_mle():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "mle_alg1.json")))
    return {(c["m"], c["profile"], c["seed"]): max(c["rel_dev"]) for c in g["cases"]}


@pytest.mark.parametrize("m,nb,profile,seeds", [(40, 200, False, (5, 6, 7, 8, 9)),
                                                (40, 200, True, (5, 6, 7, 8, 9)),
                                                (80, 400, False, (5, 6, 7))])
def test_mixed_precision_mle_matches_fp64(G, m, nb, profile, seeds):
    golden = _golden_mle()
    devs, alg1 = [], []
    for seed in seeds:
        x, y, z = grid_problem(m, seed, (1.0, 0.1, 0.5))
        X, Y, Z = dev(x), dev(y), dev(z)
        th0 = G.Theta(0.5, 0.05, 0.5)
        kw = dict(max_evals=500, xtol=1e-7, profile=profile)
        ref = G.TileStore(m * m, nb, 100, G.GEO_LP_SPLIT_BF16).mle(X, Y, Z, th0, **kw)   # all tiles FP64
        mp = G.TileStore(m * m, nb, 1, G.GEO_LP_SPLIT_BF16).mle(X, Y, Z, th0, **kw)
        d = max(rel(getattr(mp["theta"], a), getattr(ref["theta"], a)) for a in ("sigma2", "beta", "nu"))
        a1 = golden[(m, profile, seed)]
        devs.append(d)
        alg1.append(a1)
        assert d <= 3.0 * a1 + 1e-3, (seed, d, a1)
    med = float(np.median(devs))
    if m == 40:
        assert med <= 1e-3, (devs, alg1)
    else:
        assert med <= 2.0 * float(np.median(alg1)), (devs, alg1)
    print(f"n={m * m} profile={profile}: GPU deviations {devs}, oracle Algorithm 1 deviations {alg1}")


def _ar1_field(x, sigma2, beta, seed):
    w = inputs.white_noise(len(x), seed)
    z = np.empty(len(x))
    z[0] = math.sqrt(sigma2) * w[0]
    rho = np.exp(-np.diff(x) / beta)
    for i in range(1, len(x)):
        z[i] = rho[i - 1] * z[i - 1] + math.sqrt(sigma2 * (1.0 - rho[i - 1] ** 2)) * w[i]
    return z


def test_fp64_mle_markov_1d_closed_form(G):
    from scipy.optimize import minimize_scalar
    n = 3000
    x, y = inputs.line_points(n, seed=31, min_gap=0.02)
    z = _ar1_field(x, 1.3, 0.08, seed=32)
    d = np.diff(x)

    def q1_ld1(beta):
        rho = np.exp(-d / beta)
        one_m = -np.expm1(-2 * d / beta)
        ld = math.fsum(np.log(one_m).tolist())
        q = z[0] ** 2 + math.fsum(((z[1:] - rho * z[:-1]) ** 2 / one_m).tolist())
        return q, ld

    def neg_profile(lb):
        q, ld = q1_ld1(math.exp(lb))
        return 0.5 * n * math.log(q / n) + 0.5 * ld

    grid = np.linspace(math.log(1e-3), math.log(2.0), 300)
    j = int(np.argmin([neg_profile(g) for g in grid]))
    res = minimize_scalar(neg_profile, bounds=(grid[j - 1], grid[j + 1]), method="bounded",
                          options={"xatol": 1e-12})
    b_hat = math.exp(res.x)
    s2_hat = q1_ld1(b_hat)[0] / n
    ts = G.TileStore(n, 500, 100, G.GEO_LP_FP32)
    got = ts.mle(dev(x), dev(y), dev(z), G.Theta(0.5, 0.05, 0.5), max_evals=400, xtol=1e-9, profile=True,
                 fix_nu=True)
    assert rel(got["theta"].beta, b_hat) <= 1e-6
    assert rel(got["theta"].sigma2, s2_hat) <= 1e-6


def test_mle_journal_resume_equals_one_run(G):
    """geo_mle's evaluation journal: the estimate run in chunks of 15
    evaluations, each chunk replaying the journal of the previous ones, ends at
    the same theta-hat (bit for bit), with the same evaluation and iteration
    counts, as one uninterrupted run; a journal from another run is refused."""
    x, y, z = grid_problem(20, 3, (1.0, 0.1, 0.5))       # n = 400
    X, Y, Z = dev(x), dev(y), dev(z)
    th0 = G.Theta(0.5, 0.05, 0.5)
    ts = G.TileStore(400, 96, 1, G.GEO_LP_SPLIT_BF16)
    whole = ts.mle(X, Y, Z, th0, max_evals=60)
    journal = {"records": np.zeros((60, 4)), "len": 0}
    budget, calls = 0, 0
    while True:
        budget = min(60, budget + 15)
        part = ts.mle(X, Y, Z, th0, max_evals=budget, journal=journal)
        calls += 1
        assert journal["len"] == part["evals"]
        if budget >= 60 or part["evals"] < budget:
            break
    assert calls >= 2
    assert part["theta"] == whole["theta"] and part["loglik"] == whole["loglik"]
    assert part["evals"] == whole["evals"] and part["iterations"] == whole["iterations"]
    # a journal of another start point does not match the simplex
    with pytest.raises(G.GeoError) as ei:
        ts.mle(X, Y, Z, G.Theta(0.7, 0.05, 0.5), max_evals=60, journal=dict(journal))
    assert ei.value.code == -6

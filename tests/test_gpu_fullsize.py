"""Parity at the benchmark's full size, in the benchmark's launch configuration.

n = 40,000 (200 x 200 jittered grid, seed 0, Morton order), Matern sigma2 = 1,
beta = 0.1, nu = 1/2, tile 500, band 1, split-BF16 off-band products and
FP64-accurate tensor-core in-band updates (the library defaults).  The dense
oracle does not finish at this size in seconds, so the checks use outputs the
oracle computes one by one and properties that hold at any size:

  * Eq. 1: sampled rows of the generated lower triangle against the oracle's
    Matern function entry by entry (FP64 band: 1e-13 relative; FP32 tiles:
    the exact value correctly rounded up to 2^-27 relative, the bound of the
    float-pair closed-form generator).
  * Algorithm 1: sampled entries of L L' against Sigma.  Pairs inside one
    diagonal tile are formed in FP64-accurate arithmetic from the stored
    factor, so their residual is FP64 rounding (1e-12 of (|L||L'|)_ab).
    Off-band pairs carry one FP32 rounding of the tile per step (p = 80
    steps, each at most u32 (|L||L'|)_ab twice: the tile and the product) and
    the FP32 panel solve in partial sums of 16 (16 + nb/16 terms deep): the
    bound is (2p + 16 + nb/16 + 16) u32 (|L||L'|)_ab.
  * Forward solve: sampled rows of L y = Z, FP64 arithmetic on the stored
    factor: |L y - Z|_a <= n u64 (|L||y|)_a (the textbook gamma_n).
  * log-determinant 2 sum log L_aa and Q = y'y against FP64 sums of the read
    diagonal and solution (n u64 relative), and the assembly of Eq. 2.
  * all-FP64 path at n = 40,000, tile 500, on the 1D Markov closed form
    (nu = 1/2 on sorted points), |dl|/|l| <= 1e-10, and the mixed-precision
    path on the same problem within the stated 1e-6.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import geo_oracle as O  # noqa: E402
from paper_2003_05324_b300 import inputs  # noqa: E402

M, NB, BAND = 200, 500, 1
N = M * M
P = N // NB
U32 = 2.0 ** -24
U64 = 2.0 ** -53
THETA = (1.0, 0.1, 0.5, 0.0)


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_05324_b300 import geo
    return geo


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def workload():
    x, y = inputs.jittered_grid(M, seed=0)
    z = inputs.matern_field_rff(x, y, THETA[0], THETA[1], THETA[2], seed=1)
    perm = O.morton_order(x, y)
    return x[perm], y[perm], z[perm]


def sample_rows(seed=3, count=48):
    """Rows spread over the whole matrix: first and last rows of the first,
    a middle and the last tile, plus seeded random rows."""
    rng = np.random.default_rng(seed)
    fixed = [0, 1, NB - 1, NB, (P // 2) * NB + 7, N - NB, N - 2, N - 1]
    rows = np.unique(np.concatenate([fixed, rng.integers(0, N, size=count)]))
    return rows.astype(np.int64)


def test_fullsize_generation_factor_solve(G, workload):
    x, y, z = workload
    th = G.Theta(*THETA)
    oth = O.Theta(*THETA)
    R = sample_rows()
    Rt = torch.as_tensor(R, device="cuda")
    X, Y, Z = dev(x), dev(y), dev(z)
    ts = G.TileStore(N, NB, BAND, G.GEO_LP_SPLIT_BF16)

    # ---- Eq. 1, sampled rows of the lower triangle
    ts.matern(X, Y, th)
    D = ts.to_dense()
    S_rows = D.index_select(0, Rt).cpu().numpy()
    del D
    torch.cuda.empty_cache()
    for a, row in zip(R, S_rows):
        b = np.arange(a + 1)
        r = np.sqrt((x[a] - x[b]) ** 2 + (y[a] - y[b]) ** 2)
        want = O.matern(r, oth.sigma2, oth.beta, oth.nu)
        want[a] = oth.sigma2 + oth.nugget
        got = row[: a + 1]
        dp = (a // NB - b // NB) < BAND
        err = np.abs(got - want)
        assert np.all(err[dp] <= 1e-13 * np.abs(want[dp]) + 1e-15), a
        w32 = np.abs(want[~dp])
        bound = 0.5 * np.spacing(w32.astype(np.float32)).astype(np.float64) + 2.0 ** -27 * w32
        assert np.all(err[~dp] <= bound), a
        assert np.all(row[a + 1:] == 0.0)

    # ---- Algorithm 1: sampled entries of L L' against Sigma
    ts.potrf()
    D = ts.to_dense()
    L_rows = D.index_select(0, Rt).cpu().numpy()
    diag = torch.diagonal(D).cpu().numpy().copy()
    del D
    torch.cuda.empty_cache()
    assert np.all(diag > 0.0)
    absL = np.abs(L_rows)
    bound_off = (2 * P + 16 + NB / 16 + 16) * U32
    worst = {"in": 0.0, "off": 0.0}
    for ia, a in enumerate(R):
        for ib in range(ia + 1):
            b = R[ib]
            s_ab = oth.sigma2 + oth.nugget if a == b else float(
                O.matern(np.array([math.hypot(x[a] - x[b], y[a] - y[b])]), oth.sigma2, oth.beta, oth.nu)[0])
            llt = math.fsum((L_rows[ia] * L_rows[ib]).tolist())
            scale = float(absL[ia] @ absL[ib])
            rel = abs(llt - s_ab) / scale
            same_tile = (a // NB) == (b // NB)
            key = "in" if same_tile else "off"
            worst[key] = max(worst[key], rel)
            assert rel <= (1e-12 if same_tile else bound_off), (int(a), int(b), rel)

    # ---- forward solve, log-determinant, quadratic form
    ld, q, yv = ts.logdet_trsv(Z, want_y=True)
    torch.cuda.synchronize()
    yv = yv.cpu().numpy()[:N]
    for ia, a in enumerate(R):
        ly = math.fsum((L_rows[ia] * yv).tolist())
        scale = float(absL[ia] @ np.abs(yv))
        assert abs(ly - z[a]) <= N * U64 * scale, (int(a), ly, z[a])
    logs = 2.0 * np.log(diag)
    ld_ref = math.fsum(logs.tolist())
    assert abs(float(ld) - ld_ref) <= N * U64 * float(np.abs(logs).sum())
    q_ref = math.fsum((yv * yv).tolist())
    assert abs(float(q) - q_ref) <= N * U64 * q_ref

    # ---- Eq. 2 through the blocking entry point (regenerates and refactors)
    l, ld2, q2 = ts.loglik(X, Y, Z, th)
    assert ld2 == float(ld) and q2 == float(q)      # same launches, fixed reduction orders
    assert abs(l - (-0.5 * N * math.log(2 * math.pi) - 0.5 * ld2 - 0.5 * q2)) <= 1e-12 * abs(l)


def markov(x, z, s2, beta):
    """Exact l of nu = 1/2 on sorted 1D points (Markov factorization)."""
    d = np.diff(x)
    rho = np.exp(-d / beta)
    one_m = -np.expm1(-2 * d / beta)
    logdet = math.log(s2) + math.fsum(np.log(s2 * one_m).tolist())
    quad = z[0] ** 2 / s2 + math.fsum(((z[1:] - rho * z[:-1]) ** 2 / (s2 * one_m)).tolist())
    return -0.5 * len(z) * math.log(2 * math.pi) - 0.5 * logdet - 0.5 * quad


@pytest.mark.parametrize("band,gate", [(10 ** 6, 1e-10), (BAND, 1e-6)])
def test_fullsize_markov_closed_form(G, band, gate):
    # correlation length of ~80 neighbouring points: adjacent tiles are strongly
    # coupled, so the off-band tiles carry real weight in mixed precision
    x, y = inputs.line_points(N, seed=7, min_gap=0.2)
    z = inputs.white_noise(N, seed=8)
    want = markov(x, z, 1.1, 0.002)
    ts = G.TileStore(N, NB, band, G.GEO_LP_SPLIT_BF16)
    l, _, _ = ts.loglik(dev(x), dev(y), dev(z), G.Theta(1.1, 0.002, 0.5))
    assert abs(l - want) <= gate * abs(want), (l, want, abs(l - want) / abs(want))


def test_golden_dense_fp64_loglik_n22500(G):
    """Against the dense FP64 oracle value near full size: n = 22,500 (150 x 150
    jittered grid, seed 0, Morton order), tile 500, stored in
    tests/golden/loglik_n22500.json by tests/golden/make_golden.py (oracle
    calls only).  The all-FP64 GPU path (both update engines) meets the 1e-10
    gate; the mixed-precision path at bands 1, 2, 4 meets the 1e-6 gate, and
    its error is reported beside the oracle's own Algorithm 1 error."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "loglik_n22500.json")))
    x, y = inputs.jittered_grid(150, seed=0)
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=1)
    perm = O.morton_order(x, y)
    x, y, z = x[perm], y[perm], z[perm]
    X, Y, Z = dev(x), dev(y), dev(z)
    th = G.Theta(*g["theta"])
    want = g["fp64"]["loglik"]
    for mode in (G.GEO_LP_SPLIT_BF16, G.GEO_LP_FP32):
        ts = G.TileStore(len(z), g["nb"], 10 ** 6, mode)
        l = ts.loglik(X, Y, Z, th)[0]
        assert abs(l - want) <= 1e-10 * abs(want), (mode, l, want)
        del ts
    report = {}
    for band in (1, 2, 4):
        ts = G.TileStore(len(z), g["nb"], band, G.GEO_LP_SPLIT_BF16)
        l = ts.loglik(X, Y, Z, th)[0]
        err = abs(l - want) / abs(want)
        alg1 = abs(g["mp"][str(band)]["loglik"] - want) / abs(want)
        report[band] = (err, alg1)
        assert err <= 1e-6, (band, err, alg1)
        del ts
    print("n=22500 |dl|/|l| (GPU mixed precision, oracle Algorithm 1) by band:", report)


def test_golden_fp64_loglik_n40000(G):
    """The benchmark's workload (n = 40,000: 200 x 200 jittered grid, seed 0,
    Morton order; tile 500) against the oracle's values in
    tests/golden/loglik_n40000.json (tests/golden/make_golden_n40000.py,
    oracle calls only): the all-FP64 GPU path meets the 1e-10 gate.  The
    oracle's own Algorithm 1 (band 1) misses the 1e-6 gate at this size
    (|dl|/|l| = 3.0e-6: FP32 storage of 97 % of the matrix), so the
    mixed-precision GPU path is held to the gate or to the oracle's
    Algorithm 1 error on the same data, whichever is larger."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "loglik_n40000.json")))
    x, y = inputs.jittered_grid(200, seed=0)
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=1)
    perm = O.morton_order(x, y)
    x, y, z = x[perm], y[perm], z[perm]
    X, Y, Z = dev(x), dev(y), dev(z)
    th = G.Theta(*g["theta"])
    want = g["fp64"]["loglik"]
    ts = G.TileStore(len(z), g["nb"], 10 ** 6, G.GEO_LP_SPLIT_BF16)
    l = ts.loglik(X, Y, Z, th)[0]
    assert abs(l - want) <= 1e-10 * abs(want), (l, want)
    del ts
    ts = G.TileStore(len(z), g["nb"], 1, G.GEO_LP_SPLIT_BF16)
    l = ts.loglik(X, Y, Z, th)[0]
    err = abs(l - want) / abs(want)
    alg1 = abs(g["mp"]["1"]["loglik"] - want) / abs(want)
    assert err <= max(1e-6, alg1), (err, alg1)
    print("n=40000 |dl|/|l|: GPU mixed precision %.3g, oracle Algorithm 1 %.3g" % (err, alg1))

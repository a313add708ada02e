"""GPU parity of the CUDA path against the oracle, through the C ABI.

Tolerances:
  * FP64 Matern entries: 1e-13 relative (+1e-15 sigma2 absolute) -- the
    trapezoid K_nu and CUDA's exp/log each contribute ~1e-14.
  * FP32 Matern entries: computed in FP32 from coordinates pre-scaled by 1/beta
    and split into float hi + lo, so x = r/beta = xh + xl is exact to far below
    u = 2^-24.  Closed forms: e^-x, the polynomial factor and sigma2 are carried
    as float pairs (relative error below 2^-28) and rounded once, so the entry
    is the exact value correctly rounded up to 2^-27 |v|:
    |dv| <= ulp(v)/2 + 2^-27 |v|.  General nu: x^nu e^-x / norm as e^A with A
    a float pair (log and exp to 2^-29), nu and log_c both as pairs, and the
    trapezoid e^x K_nu(x) summed in pair arithmetic from terms whose only FP32
    rounding is that of their exponent a = x (cosh t - 1) (about 3u a, the
    weights decaying like e^-a): |dv| <= ulp(v)/2 + 8u |v|.
  * all-FP64 log-likelihood: |dl|/|l| <= 1e-10 (the stated gate).
  * mixed precision: |dl|/|l| <= 1e-6 against the FP64 oracle (the stated gate).
    Element-wise, the GPU's and the oracle's Algorithm 1 factors are two
    FP32-level approximations of the FP64 factor that differ in rounding order
    only; the GPU's distance to the FP64 factor must stay within twice the
    oracle's, hence (triangle inequality) within three times of the oracle's
    factor itself.  Its log-likelihood error must stay within four times the
    oracle's (plus 1e-9 relative).
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


def problem(m, seed, theta, morton=True):
    x, y = inputs.jittered_grid(m, seed=seed)
    if morton:
        perm = O.morton_order(x, y)
        x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, theta.sigma2, theta.beta, theta.nu, seed=seed + 1, nugget=theta.nugget)
    return x, y, z


def oracle_theta(th):
    return O.Theta(th.sigma2, th.beta, th.nu, th.nugget)


# ------------------------------------------------------------- A2: Eq. 1 ---
@pytest.mark.parametrize("nu", [0.5, 1.0, 1.5, 0.8, 2.5])
def test_matern_tiles_match_oracle(G, nu):
    th = G.Theta(1.3, 0.07, nu, 1e-4)
    x, y = inputs.uniform_points(700, seed=3)
    ts = G.TileStore(700, 96, 2, G.GEO_LP_FP32)   # ragged: p = 8, last tile 28 rows
    ts.matern(dev(x), dev(y), th)
    got = ts.to_dense().cpu().numpy()
    want = np.tril(O.covariance(x, y, theta=oracle_theta(th)))
    nb, band = 96, 2
    I, J = np.indices(want.shape)
    dpm = (I // nb - J // nb) < band
    lower = I >= J
    m64 = dpm & lower
    err = np.abs(got - want)
    assert np.all(err[m64] <= 1e-13 * np.abs(want[m64]) + 1e-15 * th.sigma2)
    m32 = (~dpm) & lower
    r = np.sqrt((x[I] - x[J]) ** 2 + (y[I] - y[J]) ** 2)
    xr = r / th.beta
    if nu in (0.5, 1.5, 2.5):
        bound = 0.5 * np.spacing(np.abs(want).astype(np.float32)).astype(np.float64) + 2.0 ** -27 * np.abs(want)
    else:
        bound = 0.5 * np.spacing(np.abs(want).astype(np.float32)).astype(np.float64) + 8 * 2.0 ** -24 * np.abs(want)
    viol = m32 & (err > bound)
    if viol.any():
        idx = np.argsort(-(err / bound)[viol])[:5]
        worst = [(float(xr[viol][q]), float(err[viol][q] / max(abs(want[viol][q]), 1e-300) / 2.0 ** -24))
                 for q in idx]
        raise AssertionError(f"{int(viol.sum())} FP32 entries over the bound; worst (x, ulps): {worst}")
    assert np.all(got[~lower] == 0.0)


# --------------------------------------------------- A3-A9 factor parity ---
def spd_matrix(n, seed, nu=0.5, beta=0.1, nugget=1e-3):
    x, y = inputs.uniform_points(n, seed=seed)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    return O.covariance(x, y, theta=O.Theta(1.0, beta, nu, nugget))


@pytest.mark.parametrize("n,nb", [(640, 128), (700, 96), (500, 500), (37, 64), (1536, 512), (1500, 720)])
@pytest.mark.parametrize("updates", ["fp64-pipe", "tensor"])
def test_fp64_factor_matches_oracle(G, n, nb, updates):
    # band = p: all tiles FP64.  "fp64-pipe": every update in FP64 FMA/DMMA;
    # "tensor": the in-band updates as FP64-accurate slice products on the
    # tensor cores (tile 512 and 720 take two and three 256-long parts).
    S = spd_matrix(n, seed=n)
    p = -(-n // nb)
    ts = G.TileStore(n, nb, p, G.GEO_LP_FP32 if updates == "fp64-pipe" else G.GEO_LP_SPLIT_BF16)
    ts.load_dense(dev(S.T))                      # column-major upload
    ts.potrf()
    got = ts.to_dense().cpu().numpy()
    Lo, info = O.dense_factor(S)
    assert info == 0
    assert np.max(np.abs(got - Lo)) <= 1e-12 * np.max(np.abs(Lo))


@pytest.mark.parametrize("band", [1, 3])
def test_tensor_fp64_updates_match_fp64_pipe(G, band):
    # the same mixed-precision factorization with the in-band updates on the
    # FP64 pipe and on the tensor cores: FP64-level agreement on every tile
    n, nb = 1536, 256
    S = spd_matrix(n, seed=9)
    out = []
    for flags in (G.GEO_FLAG_FP64_DMMA, 0):
        ts = G.TileStore(n, nb, band, G.GEO_LP_SPLIT_BF16)
        ts.set_flags(flags)
        ts.load_dense(dev(S.T))
        ts.potrf()
        out.append(ts.to_dense().cpu().numpy())
    Lmp, _ = O.mp_tile_cholesky(S, nb, band)
    Ldp, _ = O.dense_factor(S)
    mp_err = np.max(np.abs(Lmp - Ldp))
    for got in out:
        assert np.max(np.abs(got - Ldp)) <= 2.0 * mp_err
    # the variants differ by FP64-level rounding in the in-band tiles (which
    # can move an FP32 rounding of an off-band tile by one unit)
    assert np.max(np.abs(out[0] - out[1])) <= 0.25 * mp_err
    if band >= 3:
        # tiles (1,1) and (2,1) are updated from FP64 panels (1,0), (2,0) only:
        # FP64 parity through one tensor-core dsyrk / dgemm
        sl = np.s_[nb:3 * nb, nb:2 * nb]
        assert np.max(np.abs(out[1][sl] - Ldp[sl])) <= 1e-12 * np.max(np.abs(Ldp))


@pytest.mark.parametrize("band,lp", [(1, "fp32"), (2, "fp32"), (1, "bf16"), (3, "bf16")])
def test_mixed_factor_matches_algorithm1(G, band, lp):
    n, nb = 768, 96   # p = 8
    S = spd_matrix(n, seed=5)
    mode = G.GEO_LP_FP32 if lp == "fp32" else G.GEO_LP_SPLIT_BF16
    ts = G.TileStore(n, nb, band, mode)
    ts.load_dense(dev(S.T))
    ts.potrf()
    got = ts.to_dense().cpu().numpy()
    Lmp, info = O.mp_tile_cholesky(S, nb, band)
    Ldp, _ = O.dense_factor(S)
    assert info == 0
    ref_err = np.max(np.abs(Lmp - Ldp))
    assert ref_err > 0
    assert np.max(np.abs(got - Ldp)) <= 2.0 * ref_err
    assert np.max(np.abs(got - Lmp)) <= 3.0 * ref_err
    # in-band tiles of the first block column see no FP32 input: FP64-exact parity
    assert np.max(np.abs(got[:band * nb, :nb] - Ldp[:band * nb, :nb])) <= 1e-12


def test_not_spd_reports_failing_row(G):
    S = spd_matrix(300, seed=9)
    S[211, 211] = -1.0
    for band in (1, 5):
        ts = G.TileStore(300, 64, band, G.GEO_LP_FP32)
        ts.load_dense(dev(S.T))
        with pytest.raises(G.NotSPDError) as ei:
            ts.potrf()
        _, info = O.dense_factor(S)
        assert ei.value.info == info == 212


# ------------------------------------------------------ A10-A12: Eq. 2 ---
def test_loglik_fp64_config_n1600(G):
    # 40 x 40 jittered grid, Morton order, sigma2=1, beta=0.1, nu=0.5, Z = L w;
    # tile 200, all 8 x 8 tiles FP64
    th = G.Theta(1.0, 0.1, 0.5)
    x, y = inputs.jittered_grid(40, seed=0)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    S = O.covariance(x, y, theta=oracle_theta(th))
    Lo, _ = O.dense_factor(S)
    z = Lo @ inputs.white_noise(1600, seed=1)
    want = O.loglik_dense(x, y, z, oracle_theta(th))
    ts = G.TileStore(1600, 200, 8, G.GEO_LP_SPLIT_BF16)
    l, ld, q = ts.loglik(dev(x), dev(y), dev(z), th)
    assert abs(l - want["loglik"]) <= 1e-10 * abs(want["loglik"])
    assert abs(ld - want["logdet"]) <= 1e-10 * abs(want["logdet"])
    assert abs(q - want["quad"]) <= 1e-10 * abs(want["quad"])


@pytest.mark.parametrize("band", [1, 2, 4])
@pytest.mark.parametrize("lp", ["fp32", "bf16"])
def test_loglik_mixed_precision_gate(G, band, lp):
    # n = 1600 geometry with the n = 40,000 workload's parameters: the stated
    # gate |dl|/|l| <= 1e-6 against the FP64 oracle, generation included
    th = G.Theta(1.0, 0.1, 0.5)
    x, y, z = problem(40, 0, th)
    want = O.loglik_dense(x, y, z, oracle_theta(th))["loglik"]
    mode = G.GEO_LP_FP32 if lp == "fp32" else G.GEO_LP_SPLIT_BF16
    ts = G.TileStore(1600, 200, band, mode)
    l, _, _ = ts.loglik(dev(x), dev(y), dev(z), th)
    assert abs(l - want) / abs(want) <= 1e-6


def oracle_mp_from_matrix(S, z, nb, band):
    L, info = O.mp_tile_cholesky(S, nb, band)
    assert info == 0
    ld, q = O.factor_logdet_quad(L, z)
    return -0.5 * len(z) * math.log(2 * math.pi) - 0.5 * ld - 0.5 * q


@pytest.mark.parametrize("band", [1, 2, 4])
@pytest.mark.parametrize("lp", ["fp32", "bf16"])
def test_factor_solve_matches_algorithm1(G, band, lp):
    # Same rounded covariance on both sides: GPU potrf + log-det + solve against
    # the oracle's Algorithm 1.  A single instance's signed error is a sum of
    # many roundings of either sign (it varies ~10x between seeds for either
    # implementation), so the accuracy class is compared over four datasets:
    # the GPU's mean |dl| must stay within twice the oracle's.
    th = O.Theta(1.0, 0.1, 0.5)
    mode = G.GEO_LP_FP32 if lp == "fp32" else G.GEO_LP_SPLIT_BF16
    eg, eo = [], []
    for seed in range(4):
        x, y, z = problem(40, seed, G.Theta(1.0, 0.1, 0.5))
        S = O.covariance(x, y, theta=th)
        Ld, _ = O.dense_factor(S)
        ld, q = O.factor_logdet_quad(Ld, z)
        want = -0.5 * 1600 * math.log(2 * math.pi) - 0.5 * ld - 0.5 * q
        mp = oracle_mp_from_matrix(S, z, 200, band)
        ts = G.TileStore(1600, 200, band, mode)
        ts.load_dense(dev(S.T))
        ts.potrf()
        gld, gq, _ = ts.logdet_trsv(dev(z))
        got = -0.5 * 1600 * math.log(2 * math.pi) - 0.5 * float(gld) - 0.5 * float(gq)
        eg.append(abs(got - want))
        eo.append(abs(mp - want))
    assert np.mean(eg) <= 2.0 * np.mean(eo) + 1e-12 * 1600, (eg, eo)


@pytest.mark.parametrize("lp", ["fp32", "bf16"])
def test_offband_updates_are_unbiased(G, lp):
    # Round-to-nearest FP32 arithmetic leaves errors of either sign; a truncating
    # accumulation would bias every tile it updates.  Per off-band tile the mean
    # signed error over the mean absolute error (vs the FP64 factor) must stay
    # at the level of the oracle's Algorithm 1 (whose values here are <= 0.05).
    th = O.Theta(1.0, 0.1, 0.5)
    x, y, z = problem(40, 1, G.Theta(1.0, 0.1, 0.5))
    S = O.covariance(x, y, theta=th)
    Ld, _ = O.dense_factor(S)
    mode = G.GEO_LP_FP32 if lp == "fp32" else G.GEO_LP_SPLIT_BF16
    ts = G.TileStore(1600, 200, 1, mode)
    ts.load_dense(dev(S.T))
    ts.potrf()
    L = ts.to_dense().cpu().numpy()
    bias = []
    for i in range(2, 8):
        for j in range(1, i):
            e = L[i * 200:(i + 1) * 200, j * 200:(j + 1) * 200] - Ld[i * 200:(i + 1) * 200, j * 200:(j + 1) * 200]
            bias.append(e.mean() / np.abs(e).mean())
    assert abs(np.mean(bias)) <= 0.05, bias


@pytest.mark.parametrize("n,nb,band", [(1000, 96, 2), (50, 64, 1), (1, 16, 1), (333, 32, 3)])
def test_loglik_ragged_sizes(G, n, nb, band):
    th = G.Theta(0.8, 0.05, 1.0, 1e-4)
    x, y = inputs.uniform_points(n, seed=n)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, 0.8, 0.05, 1.0, seed=2, nugget=1e-4)
    want = O.loglik_dense(x, y, z, oracle_theta(th))["loglik"]
    mp = O.loglik_mp(x, y, z, oracle_theta(th), nb, band)["loglik"]
    p = -(-n // nb)
    ts = G.TileStore(n, nb, p, G.GEO_LP_FP32)
    l, _, _ = ts.loglik(dev(x), dev(y), dev(z), th)
    assert abs(l - want) <= 1e-10 * abs(want)
    for mode in (G.GEO_LP_FP32, G.GEO_LP_SPLIT_BF16):
        ts2 = G.TileStore(n, nb, band, mode)
        l2, _, _ = ts2.loglik(dev(x), dev(y), dev(z), th)
        assert abs(l2 - want) <= max(1e-6 * abs(want), 4 * abs(mp - want))


def test_loglik_identity_covariance_is_exact(G):
    th = G.Theta(1.0, 1e-6, 0.5)
    x, y = inputs.jittered_grid(30, seed=4)
    z = inputs.white_noise(900, seed=5)
    want = -0.5 * 900 * math.log(2 * math.pi) - 0.5 * math.fsum((z * z).tolist())
    for band in (1, 3):
        ts = G.TileStore(900, 128, band, G.GEO_LP_SPLIT_BF16)
        l, ld, q = ts.loglik(dev(x), dev(y), dev(z), th)
        assert ld == 0.0
        assert abs(l - want) <= 1e-13 * abs(want)


def markov(x, z, s2, beta):
    d = np.diff(x)
    rho = np.exp(-d / beta)
    one_m = -np.expm1(-2 * d / beta)
    logdet = math.log(s2) + math.fsum(np.log(s2 * one_m).tolist())
    quad = z[0] ** 2 / s2 + math.fsum(((z[1:] - rho * z[:-1]) ** 2 / (s2 * one_m)).tolist())
    return -0.5 * len(z) * math.log(2 * math.pi) - 0.5 * logdet - 0.5 * quad


@pytest.mark.parametrize("mode", ["fp64-pipe", "tensor"])
def test_loglik_markov_closed_form_fp64(G, mode):
    n = 6000
    x, y = inputs.line_points(n, seed=7, min_gap=0.2)
    z = inputs.white_noise(n, seed=8)
    want = markov(x, z, 1.1, 0.002)
    ts = G.TileStore(n, 500, 100, G.GEO_LP_FP32 if mode == "fp64-pipe" else G.GEO_LP_SPLIT_BF16)
    l, _, _ = ts.loglik(dev(x), dev(y), dev(z), G.Theta(1.1, 0.002, 0.5))
    assert abs(l - want) <= 1e-10 * abs(want)


@pytest.mark.parametrize("n,nb,band,flags", [(1000, 96, 2, 0), (1000, 96, 2, 4), (333, 32, 3, 0), (40, 64, 1, 0),
                                             (1536, 512, 1, 0)])
def test_fused_solve_equals_standalone_solve(G, n, nb, band, flags):
    """The forward solve run inside the factorization launch (geo_loglik,
    geo_loglik_async) performs, per element, the operations of the standalone
    geo_logdet_trsv in the same order: the two give the same bits."""
    th = G.Theta(1.0, 0.1, 0.5, 1e-6)
    x, y = inputs.uniform_points(n, seed=21)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.white_noise(n, seed=22)
    X, Y, Z = dev(x), dev(y), dev(z)
    ts = G.TileStore(n, nb, band, G.GEO_LP_SPLIT_BF16)
    ts.set_flags(flags)
    l, ld, q = ts.loglik(X, Y, Z, th)
    lda, qa, la = ts.loglik_async(X, Y, Z, th).cpu().tolist()
    ts.matern(X, Y, th)
    ts.potrf()
    lds, qs, _ = ts.logdet_trsv(Z)
    torch.cuda.synchronize()
    assert ld == float(lds) and q == float(qs)
    assert lda == ld and qa == q and la == l
    # Eq. 2 assembled on the device: the host's expression with the correctly
    # rounded log(2 pi) (one ulp above math.log(2 pi)) gives the same bits
    log2pi = float("1.8378770664093454835606594728112")
    assert la == -0.5 * n * log2pi - 0.5 * ld - 0.5 * q
    want = O.loglik_dense(x, y, z, oracle_theta(th))["loglik"]
    assert abs(l - want) <= 1e-6 * abs(want)


def test_async_result_is_nan_when_not_spd(G):
    """A factorization that meets a non-positive pivot leaves NaN in all three
    device results of geo_loglik_async (never the values of an earlier call on
    the same buffer), and the status words report it.  The failing case is the
    DST truncation whose matrix is indefinite (smallest eigenvalue -0.35)."""
    x, y = inputs.jittered_grid(40, seed=0)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.white_noise(len(x), seed=1)
    X, Y, Z = dev(x), dev(y), dev(z)
    ts = G.TileStore(len(z), 200, 3, G.GEO_LP_SPLIT_BF16)
    ts.set_flags(G.GEO_FLAG_DST)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    ts.loglik_async(X, Y, Z, G.Theta(1.0, 0.03, 0.5), out=out)
    assert np.all(np.isfinite(out.cpu().numpy()))
    ts.loglik_async(X, Y, Z, G.Theta(1.0, 0.03, 1.0), out=out)
    code, _ = ts.status()
    assert code == G.GEO_ERR_NOT_SPD
    assert np.all(np.isnan(out.cpu().numpy()))


def test_standalone_solve_is_nan_after_failed_factor(G):
    """geo_logdet_trsv on a store whose factorization failed writes NaN."""
    S = spd_matrix(300, seed=9)
    S[211, 211] = -1.0
    ts = G.TileStore(300, 64, 1, G.GEO_LP_FP32)
    ts.load_dense(dev(S.T))
    with pytest.raises(G.NotSPDError):
        ts.potrf()
    ld, q, _ = ts.logdet_trsv(dev(np.ones(300)))
    assert math.isnan(float(ld)) and math.isnan(float(q))


def test_loglik_deterministic(G):
    th = G.Theta(1.0, 0.1, 1.0)
    x, y, z = problem(30, 3, th)
    ts = G.TileStore(900, 128, 2, G.GEO_LP_SPLIT_BF16)
    a = ts.loglik(dev(x), dev(y), dev(z), th)
    b = ts.loglik(dev(x), dev(y), dev(z), th)
    assert a == b


# ------------------------------------------------------------ A13: kriging ---
@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_krige_matches_oracle(G, nu):
    th = G.Theta(1.0, 0.1, nu, 1e-6)
    x, y = inputs.uniform_points(1200, seed=11)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, nu, seed=12)
    xn, yn = inputs.uniform_points(40, seed=13)
    want = O.krige(x, y, z, oracle_theta(th), xn, yn)
    ts = G.TileStore(1200, 128, 10, G.GEO_LP_FP32)
    ts.matern(dev(x), dev(y), th)
    ts.potrf()
    got = ts.krige(dev(x), dev(y), dev(z), th, dev(xn), dev(yn)).cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-9)


def test_module_level_api(G):
    # geo.loglik on a fresh store equals the store's own evaluation bit for bit;
    # geo.Server is the serving loop
    x, y = inputs.jittered_grid(30, seed=3)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.white_noise(len(x), seed=4)
    X, Y, Z = (torch.as_tensor(v, device="cuda") for v in (x, y, z))
    th = G.Theta(1.0, 0.1, 0.5)
    want = G.TileStore(len(z), 128, 2, G.GEO_LP_SPLIT_BF16).loglik(X, Y, Z, th)[0]
    assert G.loglik(X, Y, Z, th, nb=128, band=2) == want
    from paper_2003_05324_b300 import serve
    assert G.Server is serve.Server


# ------------------------------ far tier (three-precision extension) ---
@pytest.mark.parametrize("products,far_band,far_dist", [(3, 3, 0.0), (1, 4, 0.0), (3, 0, 0.25)])
def test_far_tier_factor_matches_oracle_emulation(G, products, far_band, far_dist):
    """Off-band tiles of the far tier are updated with 3 or 1 slice products.
    The oracle's Algorithm 1 with the same far-tile map and its exact-integer
    emulation of those products (far_product) is the reference: the GPU factor
    stays within three times the FP32 tier's own error of it everywhere, while
    the far tier itself moves the factor away from FP64 by more than that (so
    the comparison sees the reduced products, not FP32 rounding).  The map
    is the oracle's own (band rule, or bounding-box distance)."""
    n, nb = 1536, 128   # p = 12
    x, y = inputs.uniform_points(n, seed=5)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    S = O.covariance(x, y, theta=O.Theta(1.0, 0.1, 0.5, 1e-3))
    far = O.far_tile_mask(x, y, nb, far_band=far_band or None, far_dist=far_dist or None)
    far &= ~np.eye(far.shape[0], dtype=bool)
    assert far.any()
    ts = G.TileStore(n, nb, 1, G.GEO_LP_SPLIT_BF16)
    ts.load_dense(dev(S.T))
    ts.set_far(far_band, dev(x), dev(y), far_dist, products)
    ts.potrf()
    got = ts.to_dense().cpu().numpy()
    Lfar, info = O.mp_tile_cholesky(S, nb, 1, far=far, far_products=products)
    assert info == 0
    Lmp, _ = O.mp_tile_cholesky(S, nb, 1)
    Ldp, _ = O.dense_factor(S)
    ref_err = np.max(np.abs(Lmp - Ldp))                # the FP32 tier's rounding
    far_err = np.max(np.abs(Lfar - Ldp))
    assert far_err > 3.0 * ref_err                     # the far tier is visible
    # Three products (20-bit slices): within the FP32 tier's own error.  One
    # product (8-bit slices): a slice of a solved panel row can round to the
    # neighbouring integer under FP32-level differences between the two
    # implementations' panel solves, a 2^-8 step of that product term; the GPU
    # must still reproduce the tier's departure from FP64 to 2 %.
    tol = 3.0 * ref_err if products == 3 else max(3.0 * ref_err, 0.02 * far_err)
    assert np.max(np.abs(got - Lfar)) <= tol
    # tiles that are not far and see no far input before step 1 are untouched by the tier
    assert np.max(np.abs(got[:, :nb] - Lmp[:, :nb])) <= 3.0 * ref_err
    # off again: the store gives the FP32-accurate tier's factor
    ts.set_far(0, None, None, 0.0, 3)
    ts.load_dense(dev(S.T))
    ts.potrf()
    assert np.max(np.abs(ts.to_dense().cpu().numpy() - Lmp)) <= 3.0 * ref_err


def test_far_tier_loglik_and_refusals(G):
    """geo_loglik on a store with a far tier, against the oracle's Algorithm 1
    with the same far map (Eq. 2 within 4x the FP32 tier's error of it plus
    1e-9), and the modes that cannot run it refuse it."""
    m, nb = 40, 200
    x, y = inputs.jittered_grid(m, seed=11)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=12)
    th = G.Theta(1.0, 0.1, 0.5)
    ts = G.TileStore(len(z), nb, 1, G.GEO_LP_SPLIT_BF16)
    ts.set_far(3, None, None, 0.0, 3)
    l = ts.loglik(dev(x), dev(y), dev(z), th)[0]
    far = O.far_tile_mask(x, y, nb, far_band=3)
    want = O.loglik_mp(x, y, z, oracle_theta(th), nb, 1, far=far, far_products=3)["loglik"]
    mp = O.loglik_mp(x, y, z, oracle_theta(th), nb, 1)["loglik"]
    dp = O.loglik_dense(x, y, z, oracle_theta(th))["loglik"]
    assert abs(l - want) <= 4.0 * abs(mp - dp) + 1e-9 * abs(dp)
    t32 = G.TileStore(len(z), nb, 1, G.GEO_LP_FP32)
    with pytest.raises(G.GeoError):
        t32.set_far(3, None, None, 0.0, 3)
    with pytest.raises(G.GeoError):
        ts.set_far(3, None, None, 0.0, 2)

"""The DST / IND approximation (Section V-B) on the GPU against the oracle.

Tiles at tile distance >= d are zero and get no tasks; the kept tiles are
FP64 and the in-band updates FP64-accurate, so the result is the oracle's
float64 Eq. 2 of the zeroed matrix up to FP64 rounding (1e-10 relative, the
all-FP64 gate).  Truncation can leave the matrix indefinite; the parameters of
the parity cases keep it positive definite (smallest eigenvalue 0.07 to 0.45,
checked with the oracle), and one case that is clearly indefinite (smallest
eigenvalue -0.35) must report GEO_ERR_NOT_SPD.
"""
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


def grid(m, seed=0):
    x, y = inputs.jittered_grid(m, seed=seed)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    return x, y, inputs.white_noise(len(x), seed=seed + 1)


def dst_store(G, n, nb, d):
    ts = G.TileStore(n, nb, d, G.GEO_LP_SPLIT_BF16)
    ts.set_flags(G.GEO_FLAG_DST)
    return ts


@pytest.mark.parametrize("m,nb,d,theta", [
    (40, 200, 1, (1.0, 0.1, 0.5, 0.0)),     # IND: independent 200-point blocks
    (40, 200, 2, (1.0, 0.03, 0.5, 0.0)),
    (40, 200, 3, (1.0, 0.03, 0.5, 0.0)),
    (40, 200, 2, (1.0, 0.02, 1.0, 0.0)),    # K_1 path
    (32, 96, 2, (1.2, 0.03, 0.5, 0.0)),     # n = 1024: ragged last tile of 64 rows
    (50, 500, 3, (1.0, 0.02, 0.5, 0.0)),    # tiles of 500: the 32-row split FP64 panel solve
])
def test_dst_loglik_matches_oracle(G, m, nb, d, theta):
    x, y, z = grid(m)
    want = O.loglik_dst(x, y, z, O.Theta(*theta), nb, d)
    assert want["info"] == 0
    ts = dst_store(G, len(z), nb, d)
    l, ld, q = ts.loglik(dev(x), dev(y), dev(z), G.Theta(*theta))
    assert abs(ld - want["logdet"]) <= 1e-10 * abs(want["logdet"])
    assert abs(q - want["quad"]) <= 1e-10 * abs(want["quad"])
    assert abs(l - want["loglik"]) <= 1e-10 * abs(want["loglik"])


def test_dst_tiles_beyond_the_band_are_zero_and_the_factor_keeps_the_band(G):
    x, y, z = grid(24)                      # n = 576, tile 96, p = 6
    n, nb, d = len(z), 96, 2
    th = G.Theta(1.0, 0.03, 0.5)
    ts = dst_store(G, n, nb, d)
    ts.matern(dev(x), dev(y), th)
    S = ts.to_dense().cpu().numpy()
    blk = np.arange(n) // nb
    far = (blk[:, None] - blk[None, :]) >= d
    assert np.all(S[far] == 0.0)
    ref = np.tril(O.dst_covariance(O.covariance(x, y, theta=O.Theta(1.0, 0.03, 0.5)), nb, d))
    assert np.allclose(S, ref, rtol=1e-13, atol=1e-15)
    ts.potrf()
    L = ts.to_dense().cpu().numpy()
    assert np.all(L[far] == 0.0)            # no fill beyond the band
    Lref, info = O.dense_factor(O.dst_covariance(O.covariance(x, y, theta=O.Theta(1.0, 0.03, 0.5)), nb, d))
    assert info == 0
    assert np.max(np.abs(L - Lref)) <= 1e-12 * np.max(np.abs(Lref))


def test_dst_band1_equals_the_sum_of_block_likelihoods(G):
    # IND identity on the GPU: one DST launch against one full evaluation per block
    x, y, z = grid(30)                      # n = 900, tile 128: blocks of 128 and a last one of 4
    n, nb = len(z), 128
    th = G.Theta(0.9, 0.08, 1.0)
    l, _, _ = dst_store(G, n, nb, 1).loglik(dev(x), dev(y), dev(z), th)
    parts = []
    for a in range(0, n, nb):
        b = min(n, a + nb)
        t = G.TileStore(b - a, nb, 1, G.GEO_LP_SPLIT_BF16)
        parts.append(t.loglik(dev(x[a:b]), dev(y[a:b]), dev(z[a:b]), th)[0])
    assert abs(l - sum(parts)) <= 1e-11 * abs(l)


def test_dst_indefinite_truncation_reports_not_spd(G):
    x, y, z = grid(40)
    ts = dst_store(G, len(z), 200, 3)
    with pytest.raises(G.NotSPDError):
        ts.loglik(dev(x), dev(y), dev(z), G.Theta(1.0, 0.03, 1.0))
    # the store stays usable: a positive definite problem afterwards
    l, _, _ = ts.loglik(dev(x), dev(y), dev(z), G.Theta(1.0, 0.03, 0.5))
    want = O.loglik_dst(x, y, z, O.Theta(1.0, 0.03, 0.5), 200, 3)["loglik"]
    assert abs(l - want) <= 1e-10 * abs(want)


def test_dst_flag_combinations_are_refused(G):
    ts = G.TileStore(400, 100, 2, G.GEO_LP_SPLIT_BF16)
    for bad in (G.GEO_FLAG_DST | G.GEO_FLAG_FP64_DMMA, G.GEO_FLAG_DST | G.GEO_FLAG_STEPWISE):
        with pytest.raises(G.GeoError):
            ts.set_flags(bad)
    t32 = G.TileStore(400, 100, 2, G.GEO_LP_FP32)
    with pytest.raises(G.GeoError):
        t32.set_flags(G.GEO_FLAG_DST)


def test_dst_in_a_batch_equals_the_single_problem(G):
    # DST problems next to an ordinary mixed-precision one in the same launch
    probs, thetas, want = [], [], []
    for s, (m, nb, d, flags) in enumerate([(30, 128, 1, G.GEO_FLAG_DST), (36, 128, 2, G.GEO_FLAG_DST),
                                           (24, 128, 2, 0), (20, 64, 3, G.GEO_FLAG_DST)]):
        x, y, z = grid(m, seed=10 + s)
        th = G.Theta(1.0, 0.02, 0.5)
        probs.append(dict(x=dev(x), y=dev(y), z=dev(z), nb=nb, band=d, flags=flags))
        thetas.append(th)
        ts = G.TileStore(len(z), nb, d, G.GEO_LP_SPLIT_BF16)
        if flags:
            ts.set_flags(flags)
        want.append(ts.loglik(dev(x), dev(y), dev(z), th))
    B = G.Batch(probs)
    got = B.loglik(thetas)
    for g, w in zip(got, want):
        assert tuple(g) == tuple(w)


def test_dst_fused_solve_sums_every_block_row(G):
    # with independent blocks nothing but the finishing rule orders the last
    # diagonal solve after the others: repeat a 20-block evaluation
    x, y, z = grid(50, seed=7)              # n = 2,500, tile 128: 20 blocks, the last of 68 rows
    th = G.Theta(1.0, 0.05, 0.5)
    want = O.loglik_dst(x, y, z, O.Theta(1.0, 0.05, 0.5), 128, 1)["loglik"]
    ts = dst_store(G, len(z), 128, 1)
    X, Y, Z = dev(x), dev(y), dev(z)
    for _ in range(10):
        l, _, _ = ts.loglik(X, Y, Z, th)
        assert abs(l - want) <= 1e-10 * abs(want)


@pytest.mark.parametrize("nb,d,theta", [
    (200, 1, (1.0, 0.1, 0.5, 0.0)),      # IND: kriging from the home block alone
    (200, 2, (1.0, 0.03, 0.5, 0.0)),
    (96, 3, (1.2, 0.02, 1.0, 1e-6)),     # ragged last tile, K_1 path (smallest eigenvalue 0.10)
])
def test_dst_krige_matches_oracle(G, nb, d, theta):
    """Kriging under the DST approximation: the new location's covariances
    are truncated like the observed ones (kept within d tiles of the tile of
    its nearest observed point); against oracle.krige_dst to 1e-8, and a new
    location on an observed one gets its observation back."""
    x, y, z = grid(40 if nb == 200 else 32)
    xn, yn = inputs.uniform_points(25, seed=31)
    xn = np.concatenate([xn, x[[0, 500, len(x) - 1]]])
    yn = np.concatenate([yn, y[[0, 500, len(x) - 1]]])
    th = O.Theta(*theta)
    want = O.krige_dst(x, y, z, th, xn, yn, nb, d)
    ts = dst_store(G, len(z), nb, d)
    ts.matern(dev(x), dev(y), G.Theta(*theta))
    ts.potrf()
    got = ts.krige(dev(x), dev(y), dev(z), G.Theta(*theta), dev(xn), dev(yn)).cpu().numpy()
    assert np.allclose(got, want, rtol=1e-8, atol=1e-10 * np.abs(want).max()), np.abs(got - want).max()
    if theta[3] == 0.0:
        np.testing.assert_allclose(got[-3:], z[[0, 500, len(x) - 1]], atol=1e-7)

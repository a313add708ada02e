"""Failure detection of the persistent scheduler without faulting the device.

Every wait inside the factorization kernel is bounded (geo_tiles_set_timeout_ns).
The test hook GEO_FLAG_TEST_STALL makes the first step's tensor-core update
items wait for a dependency count that the factorization never reaches; with a 50 ms bound the
launch must end by itself with GEO_ERR_TIMEOUT and the wait's location code,
leave NaN in the results, return its tensor memory, and the same store (and
the device) must then give the correct likelihood again.
"""
import math
import time

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


def problem(m=40, seed=3):
    x, y = inputs.jittered_grid(m, seed=seed)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=seed + 1)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    return x, y, z, d(x), d(y), d(z)


def test_timeout_bound_is_validated(G):
    ts = G.TileStore(400, 100, 1, G.GEO_LP_SPLIT_BF16)
    for bad in (1, 99_999, 10 ** 13, -5):
        with pytest.raises(G.GeoError):
            ts.set_timeout_ns(bad)
    ts.set_timeout_ns(50_000_000)
    ts.set_timeout_ns(0)


@pytest.mark.parametrize("nb,band", [(200, 1), (128, 2)])
def test_stalled_dependency_times_out_and_store_recovers(G, nb, band):
    x, y, z, X, Y, Z = problem()
    th = G.Theta(1.0, 0.1, 0.5)
    ts = G.TileStore(len(z), nb, band, G.GEO_LP_SPLIT_BF16)
    good = ts.loglik_async(X, Y, Z, th).cpu().numpy()
    assert np.all(np.isfinite(good))
    ts.set_flags(G.GEO_FLAG_TEST_STALL)
    ts.set_timeout_ns(50_000_000)                    # 50 ms per wait
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = ts.loglik_async(X, Y, Z, th).cpu().numpy()
    wall = time.perf_counter() - t0
    code, where = ts.status()
    assert code == G.GEO_ERR_TIMEOUT and where == 31, (code, where)
    assert np.all(np.isnan(res))
    assert wall < 5.0                                 # ended by the bound, not by luck
    # the blocking call reports the same failure
    with pytest.raises(G.GeoError) as ei:
        ts.loglik(X, Y, Z, th)
    assert ei.value.code == G.GEO_ERR_TIMEOUT
    # hook cleared, default bound: the same store gives the same bits as before
    ts.set_flags(0)
    ts.set_timeout_ns(0)
    again = ts.loglik_async(X, Y, Z, th).cpu().numpy()
    assert ts.status()[0] == G.GEO_OK
    assert np.array_equal(again, good)
    want = O.loglik_dense(x, y, z, O.Theta(1.0, 0.1, 0.5))["loglik"]
    assert abs(again[2] - want) <= 1e-6 * abs(want)


def test_other_stores_unaffected_after_a_timeout(G):
    """A timeout in one store's launch leaves the device usable: a fresh
    all-FP64 store afterwards matches the oracle to the FP64 gate."""
    x, y, z, X, Y, Z = problem(m=30, seed=5)
    ts = G.TileStore(len(z), 100, 1, G.GEO_LP_SPLIT_BF16)
    ts.set_flags(G.GEO_FLAG_TEST_STALL)
    ts.set_timeout_ns(20_000_000)
    ts.loglik_async(X, Y, Z, G.Theta(1.0, 0.1, 0.5))
    assert ts.status()[0] == G.GEO_ERR_TIMEOUT
    t64 = G.TileStore(len(z), 100, 100, G.GEO_LP_SPLIT_BF16)
    l = t64.loglik(X, Y, Z, G.Theta(1.0, 0.1, 0.5))[0]
    want = O.loglik_dense(x, y, z, O.Theta(1.0, 0.1, 0.5))["loglik"]
    assert math.isfinite(l) and abs(l - want) <= 1e-10 * abs(want)

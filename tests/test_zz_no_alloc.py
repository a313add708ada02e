"""The allocation-free log-det / forward-solve entry point.

geo_logdet_trsv_noalloc serves callers that cannot allocate device memory
(code running during CUDA graph capture, or frameworks whose pool owns the
device): its scratch is a fixed array inside the library.  Checked here through
the C ABI against geo_logdet_trsv (which takes its scratch from the caller's
workspace) on the same factored store, on two calls in a row, plus the size
limit.  This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_05324_b300 import geo
    return geo


def _problem(G):
    from paper_2003_05324_b300 import inputs
    x, y = inputs.jittered_grid(45, seed=7)   # n = 2025, tile 200 -> 11 x 11 tiles, ragged last tile
    perm = G.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, 1.0, 0.1, 0.5, seed=8)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    return d(x), d(y), d(z), len(z)


def _call(G, fn, ts, Z, *extra):
    ld = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    q = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = int(torch.cuda.current_stream().cuda_stream)
    rc = fn(ctypes.byref(ts.t), Z.data_ptr(), ld.data_ptr(), q.data_ptr(), *extra, stream)
    assert rc == G.GEO_OK
    torch.cuda.synchronize()
    return float(ld.item()), float(q.item())


@pytest.mark.parametrize("lp", ["bf16", "fp32"])
def test_noalloc_matches_workspace_solve_twice(G, lp):
    X, Y, Z, n = _problem(G)
    th = G.Theta(1.0, 0.1, 0.5)
    ts = G.TileStore(n, 200, 1, G.GEO_LP_SPLIT_BF16 if lp == "bf16" else G.GEO_LP_FP32)
    ts.matern(X, Y, th)
    ts.potrf()
    ref_ld, ref_q = _call(G, G.lib.geo_logdet_trsv, ts, Z, None)
    assert math.isfinite(ref_ld) and math.isfinite(ref_q)
    for _ in range(2):
        ld, q = _call(G, G.lib.geo_logdet_trsv_noalloc, ts, Z)
        # same kernels on the same data: equal within the tests' FP64 tolerance
        assert abs(ld - ref_ld) <= 1e-12 * abs(ref_ld)
        assert abs(q - ref_q) <= 1e-12 * abs(ref_q)


def test_noalloc_rejects_sizes_beyond_its_buffer(G):
    X, Y, Z, n = _problem(G)
    ts = G.TileStore(n, 200, 1, G.GEO_LP_FP32)
    big = G.geo_tiles()
    ctypes.memmove(ctypes.byref(big), ctypes.byref(ts.t), ctypes.sizeof(G.geo_tiles))
    big.lay.p = G.GEO_NOALLOC_MAX_N // 200 + 1      # p * nb just above the limit; nothing is launched
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = G.lib.geo_logdet_trsv_noalloc(ctypes.byref(big), Z.data_ptr(), ld.data_ptr(), ld.data_ptr(), None)
    assert rc == G.GEO_ERR_TOO_LARGE


def test_noalloc_after_failed_factor_is_nan_not_stale(G):
    """A call on a store whose factorization failed must not return the partial
    sums an earlier call left in the shared array: it returns NaN."""
    X, Y, Z, n = _problem(G)
    th = G.Theta(1.0, 0.1, 0.5)
    good = G.TileStore(n, 200, 1, G.GEO_LP_FP32)
    good.matern(X, Y, th)
    good.potrf()
    ld, q = _call(G, G.lib.geo_logdet_trsv_noalloc, good, Z)
    assert math.isfinite(ld) and math.isfinite(q)
    from oracle import geo_oracle as O
    S = O.covariance(X.cpu().numpy(), Y.cpu().numpy(), theta=O.Theta(1.0, 0.1, 0.5))
    S[700, 700] = -1.0                              # not positive definite at row 701
    bad = G.TileStore(n, 200, 1, G.GEO_LP_FP32)
    bad.load_dense(torch.as_tensor(np.ascontiguousarray(S.T), device="cuda"))
    with pytest.raises(G.NotSPDError):
        bad.potrf()
    ld2, q2 = _call(G, G.lib.geo_logdet_trsv_noalloc, bad, Z)
    assert math.isnan(ld2) and math.isnan(q2)
    # the next good call is unaffected
    ld3, q3 = _call(G, G.lib.geo_logdet_trsv_noalloc, good, Z)
    assert ld3 == ld and q3 == q

"""Serving with continuous batching (paper_2003_05324_b300.serve).

* Every result served in a mix of concurrent requests equals the same request
  evaluated alone, bit for bit (log-likelihood: the single-problem path;
  kriging: a direct prediction from the resident factor).
* Continuous batching: a short request that arrives while a long one is on
  the device is admitted into the other lane at once, runs beside it and
  finishes first, and both results equal their values alone.
* HBM-budget admission: the resident kriging factors count against the
  budget; with room for one more store at a time the requests are served over
  several launches with the same results; a request whose store can never fit
  beside the resident factors is rejected, and with room for the resident
  factors only every likelihood request is rejected while kriging is served.
* Kriging from the mixed-precision resident factor: MSPE against the held-out
  truth within 1% of the FP64 path's (the stated gate), and the FP64 path's
  predictions match the oracle's to 1e-8.
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
    from paper_2003_05324_b300 import geo, serve
    return geo, serve


def dataset(n, seed, th, nb=128):
    x, y = inputs.uniform_points(n + 100, seed=seed)
    z = inputs.matern_field_rff(x, y, th[0], th[1], th[2], seed=seed + 1)
    xo, yo, zo = x[:n], y[:n], z[:n]
    perm = O.morton_order(xo, yo)
    return dict(x=xo[perm], y=yo[perm], z=zo[perm], nb=nb, xt=x[n:], yt=y[n:], zt=z[n:], th=th)


def make_requests(geo, serve, dss, rng):
    reqs = []
    for q in range(12):
        d = q % len(dss)
        if q % 3 == 2:
            reqs.append(serve.Request("krige", d, xnew=dss[d]["xt"], ynew=dss[d]["yt"], t_arrival=0.0, id=q))
        else:
            th = dss[d]["th"]
            reqs.append(serve.Request("loglik", d, theta=geo.Theta(th[0] * rng.uniform(0.7, 1.3),
                                                                   th[1] * rng.uniform(0.7, 1.3), th[2]),
                                      t_arrival=0.0, id=q))
    return reqs


@pytest.fixture(scope="module")
def dss():
    return [dataset(600, 1, (1.0, 0.1, 0.5)), dataset(900, 2, (1.3, 0.05, 1.5)),
            dataset(1300, 3, (0.8, 0.08, 0.5)), dataset(2000, 4, (1.0, 0.1, 1.0), nb=256)]


def server(geo, serve, dss, budget, lanes=2):
    return serve.Server([dict(x=d["x"], y=d["y"], z=d["z"], theta=geo.Theta(*d["th"]), nb=d["nb"]) for d in dss],
                        hbm_budget_bytes=budget, lanes=lanes)


def resident(serve, dss):
    return sum(serve.store_bytes(len(d["z"]), d["nb"], 1) for d in dss)


def alone(geo, S, r):
    d = S.ds[r.dataset]
    if r.kind == "loglik":
        ts = geo.TileStore(d["n"], d["nb"], 1, geo.GEO_LP_SPLIT_BF16)
        return tuple(ts.loglik(d["x"], d["y"], d["z"], r.theta))
    xn = torch.as_tensor(r.xnew, device="cuda")
    yn = torch.as_tensor(r.ynew, device="cuda")
    return d["krig"].krige(d["x"], d["y"], d["z"], d["theta"], xn, yn).cpu().numpy()


@pytest.mark.parametrize("budget_stores,lanes", [(100, 2), (1, 2), (100, 1)])
def test_served_results_equal_alone(G, dss, budget_stores, lanes):
    geo, serve = G
    big = max(serve.store_bytes(len(d["z"]), d["nb"], 1) for d in dss)
    S = server(geo, serve, dss, resident(serve, dss) + budget_stores * big, lanes)
    reqs = make_requests(geo, serve, dss, np.random.default_rng(5))
    results, stats = S.run(reqs)
    assert stats["completed"] == len(reqs) and stats["rejected"] == 0 and stats["queued"] == 0
    if budget_stores == 1:
        assert stats["launches"] >= 2          # one store at a time: several launches
    else:
        assert stats["launches"] == 1          # everything admitted together
    byid = {r.id: r for r in results}
    for r in reqs:
        got = byid[r.id].value
        want = alone(geo, S, r)
        assert np.array_equal(np.asarray(got), np.asarray(want)), (r.kind, r.dataset)
    assert stats["p50_ms"] <= stats["p99_ms"]


def test_request_larger_than_budget_is_rejected(G, dss):
    geo, serve = G
    small = min(serve.store_bytes(len(d["z"]), d["nb"], 1) for d in dss)
    S = server(geo, serve, dss, resident(serve, dss) + small)   # beside the resident factors: the smallest store
    th = geo.Theta(*dss[3]["th"])
    results, stats = S.run([serve.Request("loglik", 3, theta=th, id=0),
                            serve.Request("loglik", 0, theta=geo.Theta(*dss[0]["th"]), id=1)])
    assert stats["rejected"] == 1 and stats["loglik_completed"] == 1 and results[0].id == 1


def test_kriging_mspe_mixed_precision_within_1pct(G, dss):
    geo, serve = G
    for d in dss:
        X, Y, Z = (torch.as_tensor(d[k], device="cuda") for k in ("x", "y", "z"))
        xn, yn = torch.as_tensor(d["xt"], device="cuda"), torch.as_tensor(d["yt"], device="cuda")
        th = geo.Theta(*d["th"])
        n = len(d["z"])
        pred = {}
        for band in (1, 100):
            ts = geo.TileStore(n, d["nb"], band, geo.GEO_LP_SPLIT_BF16)
            ts.matern(X, Y, th)
            ts.potrf()
            pred[band] = ts.krige(X, Y, Z, th, xn, yn).cpu().numpy()
        want = O.krige(d["x"], d["y"], d["z"], O.Theta(*d["th"]), d["xt"], d["yt"])
        assert np.max(np.abs(pred[100] - want)) <= 1e-8 * np.max(np.abs(want))
        m_mp = np.mean((pred[1] - d["zt"]) ** 2)
        m_dp = np.mean((pred[100] - d["zt"]) ** 2)
        assert abs(m_mp - m_dp) <= 0.01 * m_dp, (m_mp, m_dp)


def test_budget_for_the_resident_factors_only(G, dss):
    """The resident kriging factors count against the HBM budget: with room
    for them and nothing else, likelihood requests are rejected (their stores
    can never fit) while kriging requests on the resident factors are served."""
    geo, serve = G
    S = server(geo, serve, dss, resident(serve, dss))
    assert S.allocated == S.resident_bytes
    reqs = make_requests(geo, serve, dss, np.random.default_rng(6))
    results, stats = S.run(reqs)
    nlik = sum(1 for r in reqs if r.kind == "loglik")
    assert stats["rejected"] == nlik and stats["loglik_completed"] == 0
    assert stats["krige_completed"] == len(reqs) - nlik
    assert S.allocated == S.resident_bytes       # nothing left allocated after the run


def test_request_arriving_mid_flight_finishes_first(G):
    """Continuous batching: a long likelihood request (n = 24,000) is on the
    device on one lane; a short one (n = 800) arrives 10 ms later, is admitted
    into the other lane while the long one runs, and completes first.  Both
    results equal the single-problem path bit for bit."""
    geo, serve = G
    dsets = []
    for n, nb, seed in ((24000, 500, 61), (800, 128, 62)):
        x, y = inputs.uniform_points(n, seed=seed)
        perm = O.morton_order(x, y)
        dsets.append(dict(x=x[perm], y=y[perm], z=inputs.white_noise(n, seed=seed + 1), nb=nb,
                          theta=geo.Theta(1.0, 0.1, 0.5, 1e-4), krige=False))
    S = serve.Server(dsets, hbm_budget_bytes=64 << 30, lanes=2)
    th = [geo.Theta(1.1, 0.09, 0.5, 1e-4), geo.Theta(0.9, 0.12, 0.5, 1e-4)]
    S.run([serve.Request("loglik", 0, theta=th[0], id=0), serve.Request("loglik", 1, theta=th[1], id=1)])  # pool stores
    results, stats = S.run([serve.Request("loglik", 0, theta=th[0], t_arrival=0.0, id=0),
                            serve.Request("loglik", 1, theta=th[1], t_arrival=0.010, id=1)])
    byid = {r.id: r for r in results}
    long_, short = byid[0], byid[1]
    assert short.lane != long_.lane
    assert long_.t_admit < short.t_admit < long_.t_done          # admitted while the long one was on the device
    assert short.t_done < long_.t_done                           # and finished first
    assert stats["launches_overlapping"] >= 1
    for r, q in ((long_, 0), (short, 1)):
        d = S.ds[q]
        ts = geo.TileStore(d["n"], d["nb"], 1, geo.GEO_LP_SPLIT_BF16)
        want = ts.loglik(d["x"], d["y"], d["z"], th[q])
        assert np.array_equal(np.asarray(r.value), np.asarray(want)), (q, r.value, want)

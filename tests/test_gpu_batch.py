"""Batched evaluation (geo_loglik_batch): many problems, one persistent launch.

* Every problem's (l, log|Sigma|, Q) in a batch is bit-for-bit the value the
  single-problem path (geo_loglik) gives for it: uneven n (ragged last tiles),
  tile sizes 64 / 128 / 256, bands 1 and 2, nu in {1/2, 1, 3/2}, and the
  in-band updates on the tensor cores or on the FP64 pipe.
* The same holds whatever else is in the batch (a problem alone, first, last).
* A problem that is not positive definite yields NaN and GEO_ERR_NOT_SPD in its
  own store; the others are unaffected.
* Replaying a captured CUDA graph with new parameters gives the results of a
  direct evaluation.
* Against the oracle: all-FP64 problems to 1e-10, mixed precision to 1e-6.
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


def make_problem(n, seed, th, nb, band, flags=0):
    x, y = inputs.uniform_points(n, seed=seed)
    perm = O.morton_order(x, y)
    x, y = x[perm], y[perm]
    z = inputs.matern_field_rff(x, y, th[0], th[1], th[2], seed=seed + 1)
    return dict(x=dev(x), y=dev(y), z=dev(z), nb=nb, band=band, flags=flags, theta=th, xh=x, yh=y, zh=z)


PROBLEMS = [  # n, seed, theta, nb, band, flags
    (700, 1, (1.0, 0.1, 0.5, 0.0), 128, 1, 0),
    (1500, 2, (1.5, 0.05, 1.0, 1e-6), 256, 2, 0),
    (333, 3, (0.8, 0.2, 1.5, 0.0), 64, 1, 0),
    (2048, 4, (1.0, 0.08, 0.5, 0.0), 256, 1, 4),      # in-band updates on the FP64 pipe
    (96, 5, (1.2, 0.3, 0.5, 0.0), 128, 1, 0),        # a single tile
    (1000, 6, (1.0, 0.1, 1.0, 0.0), 128, 3, 0),
]


def single(G, pr):
    ts = G.TileStore(int(pr["z"].shape[0]), pr["nb"], pr["band"], G.GEO_LP_SPLIT_BF16)
    if pr["flags"]:
        ts.set_flags(pr["flags"])
    return np.array(ts.loglik(pr["x"], pr["y"], pr["z"], G.Theta(*pr["theta"])))


@pytest.fixture(scope="module")
def probs(G):
    return [make_problem(*a) for a in PROBLEMS]


def test_batch_equals_single_problem_path_bitwise(G, probs):
    B = G.Batch(probs)
    out = B.loglik([G.Theta(*pr["theta"]) for pr in probs])
    for b, pr in enumerate(probs):
        want = single(G, pr)
        assert np.array_equal(out[b], want), (b, out[b], want)


def test_batch_result_does_not_depend_on_the_mix(G, probs):
    full = G.Batch(probs).loglik([G.Theta(*pr["theta"]) for pr in probs])
    rev = list(reversed(probs))
    out_rev = G.Batch(rev).loglik([G.Theta(*pr["theta"]) for pr in rev])
    for b in range(len(probs)):
        assert np.array_equal(out_rev[len(probs) - 1 - b], full[b])
    alone = G.Batch([probs[1]]).loglik([G.Theta(*probs[1]["theta"])])
    assert np.array_equal(alone[0], full[1])


def test_not_spd_problem_is_isolated(G, probs):
    # a negative nugget makes the first pivot sigma2 + nugget < 0 (theta in
    # device memory is not validated by the batched path)
    bad = make_problem(500, 9, (1.0, 0.1, 0.5, -2.0), 128, 1)
    mix = [probs[0], bad, probs[2]]
    B = G.Batch(mix)
    out = B.loglik([G.Theta(*pr["theta"]) for pr in mix])
    assert np.all(np.isnan(out[1]))
    code, info = B.status()[1]
    assert code == G.GEO_ERR_NOT_SPD and info == 1
    assert np.array_equal(out[0], single(G, probs[0]))
    assert np.array_equal(out[2], single(G, probs[2]))


def test_graph_replay_with_new_parameters(G, probs):
    B = G.Batch(probs)
    th0 = [G.Theta(*pr["theta"]) for pr in probs]
    B.loglik(th0)
    B.capture()
    th1 = [G.Theta(t.sigma2 * 1.3, t.beta * 0.9, t.nu, t.nugget) for t in th0]
    got = B.replay(th1)
    want = G.Batch(probs).loglik(th1)
    assert np.array_equal(got, want)
    assert np.array_equal(B.replay(th0), G.Batch(probs).loglik(th0))


def test_batch_against_the_oracle(G):
    prs = [make_problem(400, 11, (1.0, 0.1, 0.5, 0.0), 64, 100),      # all FP64
           make_problem(640, 12, (1.3, 0.07, 1.0, 0.0), 128, 100),
           make_problem(900, 13, (1.0, 0.1, 0.5, 0.0), 128, 1),       # mixed precision
           make_problem(1200, 14, (0.9, 0.05, 1.5, 0.0), 256, 1)]
    out = G.Batch(prs).loglik([G.Theta(*pr["theta"]) for pr in prs])
    for b, pr in enumerate(prs):
        want = O.loglik_dense(pr["xh"], pr["yh"], pr["zh"], O.Theta(*pr["theta"]))["loglik"]
        tol = 1e-10 if pr["band"] >= 100 else 1e-6
        assert abs(out[b][0] - want) <= tol * abs(want), (b, out[b][0], want)


def test_per_problem_completion_stamps(G):
    """Each problem's solve runs inside the batched launch and stamps its
    completion: every stamp lies after the launch start, a problem of 4 tiles
    finishes before one of 24 tiles in the same launch, and the results equal
    the single-problem path bit for bit."""
    small = make_problem(500, 11, (1.0, 0.1, 0.5, 0.0), 128, 1)
    big = make_problem(6000, 12, (1.0, 0.1, 0.5, 0.0), 256, 1)
    B = G.Batch([small, big])
    out = B.loglik([G.Theta(*small["theta"]), G.Theta(*big["theta"])])
    t = B.done_ns.cpu().numpy()
    assert t[0] > 0 and np.all(t[1:] > t[0])
    ms = B.completion_ms()
    assert ms[0] < ms[1], ms
    assert np.array_equal(out[0], single(G, small)) and np.array_equal(out[1], single(G, big))


@pytest.mark.parametrize("ctas", [16, 4])
def test_partial_sm_launch_equals_full(G, probs, ctas):
    """A launch on a share of the SMs (geo_batch_set_ctas, a plain launch) gives
    the same bits as the cooperative launch on every SM, down to GEO_MIN_CTAS
    CTAs, with FP64 bulk items in the batch (the problem with the in-band updates
    on the FP64 pipe) and without."""
    full = G.Batch(probs).loglik([G.Theta(*pr["theta"]) for pr in probs])
    part = G.Batch(probs, ctas=ctas).loglik([G.Theta(*pr["theta"]) for pr in probs])
    assert not np.isnan(full).any()
    assert np.array_equal(full, part, equal_nan=True)
    tensor_only = [pr for pr in probs if not pr["flags"]]
    assert len(tensor_only) < len(probs)
    full = G.Batch(tensor_only).loglik([G.Theta(*pr["theta"]) for pr in tensor_only])
    part = G.Batch(tensor_only, ctas=ctas).loglik([G.Theta(*pr["theta"]) for pr in tensor_only])
    assert np.array_equal(full, part, equal_nan=True)

"""Host-side logic of the study and profiling tools (no GPU): the accuracy
study's summary and resume bookkeeping, and the task-trace summary."""
import json

import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2003_05324_b300 import accuracy_study as S  # noqa: E402
from paper_2003_05324_b300 import run  # noqa: E402


def row(beta, seed, method, th, mspe, evals=100, iters=50):
    return {"theta2": beta, "seed": seed, "method": method, "n": 1600, "theta_hat": th, "loglik": 0.0,
            "evals": evals, "iterations": iters, "not_spd_evals": 0, "seconds": 1.0, "cv_folds": 10, "mspe": mspe}


def test_study_summary_distances_and_ratios():
    rows = [row(0.1, 0, "DP", [1.0, 0.1, 0.5], 2.0), row(0.1, 1, "DP", [2.0, 0.2, 0.5], 4.0),
            row(0.1, 0, "MP b=1", [1.01, 0.1, 0.5], 2.0), row(0.1, 1, "MP b=1", [2.0, 0.19, 0.5], 5.0),
            {"theta2": 0.1, "seed": 0, "method": "DST d=1", "n": 1600, "status": "indefinite"}]
    out = {s["method"]: s for s in S.summary(rows, [0.1], ["DP", "MP b=1", "DST d=1"])}
    assert out["DP"]["max_rel_dist_to_dp"] == 0.0 and out["DP"]["mean_mspe_ratio_to_dp"] == 1.0
    mp = out["MP b=1"]
    assert mp["datasets"] == 2
    assert np.isclose(mp["max_rel_dist_to_dp"], 0.05)            # beta 0.19 against 0.2
    assert np.isclose(mp["median_rel_dist_to_dp"], (0.01 + 0.05) / 2)
    assert np.isclose(mp["mean_mspe_ratio_to_dp"], (1.0 + 1.25) / 2)
    assert out["DST d=1"]["status"].startswith("no estimate")


def test_study_resume_skips_done_rows(monkeypatch):
    """run_study computes only the (theta2, seed, method) rows missing from
    `done`; with all rows done it touches no device."""
    done = [row(0.1, 0, m, [1.0, 0.1, 0.5], 1.0) for m in ("DP", "MP b=1")]
    emitted = []
    monkeypatch.setattr(S, "exact_field", lambda *a, **k: pytest.fail("no dataset needed"))
    rows = S.run_study(40, 200, [0.1], [0], 10, ["DP", "MP b=1"], emit=emitted.append, done=done, dev="cpu")
    assert rows == done and emitted == []
    json.dumps(rows)


def trace_records():
    dt = np.dtype([("type", "i4"), ("sm", "i4"), ("k", "i4"), ("a", "i4"), ("b", "i4"), ("c", "i4"),
                   ("t_claim", "i8"), ("t_ready", "i8"), ("t_end", "i8")])
    recs = []
    # two SMs, each finishing an off-band item every 10 us (products done), epilogue 4 us
    for sm in (0, 1):
        for q in range(5):
            t = 1_000_000 + q * 10_000
            recs.append((10, sm, q, 0, 0, 0, t - 4_000, t, t + 4_000))
            recs.append((15, sm, q, 0, 0, 0, t - 9_000, t - 8_000, t - 1_000))   # MMA: 1 us wait, 7 us issue
            recs.append((16, sm, q, 0, 0, 0, t - 12_000, t - 10_000, t - 9_500))  # copy: 2 us, 0.5 us
    for k in range(10):                                                           # PC(k): 100 us wait, 300 us work
        t = 1_000_000 + k * 500_000
        recs.append((7, 0, k, 0, 0, 0, t, t + 100_000, t + 400_000))
    return np.array(recs, dtype=dt)


def test_trace_summary_reports_the_phases():
    lines = []
    run.summarize_trace(trace_records(), out=lines.append)
    text = "\n".join(lines)
    assert "type 10: n=      10" in text and "type  7: n=      10" in text
    assert "off-band item period per SM us: p10 10.00 p50 10.00 p90 10.00 | epilogue us p50 4.00" in text
    assert "MMA thread: wait for first stage us: p50 1.00" in text
    assert "MMA thread: first stage to last MMA us: p50 7.00" in text
    assert "copy thread: take item to dependencies met us: p50 2.00" in text
    assert "copy thread: dependencies to first copies us: p50 0.50" in text
    assert "PC(k), last 45 % of steps: wait us 100.0, work us 300.0, steps 0.500 ms apart" in text

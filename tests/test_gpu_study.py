"""The accuracy study's driver (Section VIII-D, reduced Monte-Carlo study) on a
small case: n = 1,600 (40 x 40 jittered grid), theta2 = 0.1, one seed, 60
Nelder-Mead evaluations, 10-fold cross-validated prediction.

* every method yields an estimate and a CV score, with its evaluation and
  iteration counts;
* mixed precision (band 1) reproduces the double-precision estimate to the
  MLE tolerance of Section IV-C's comparison (1e-3 relative here, where the
  two runs take the same simplex path) and its prediction error to 1 %;
* the independent-blocks approximation (DST, d = 1) predicts no better than
  the full model.
"""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_05324_b300 import accuracy_study
    return accuracy_study


def test_study_driver_small(S):
    lines = []
    rows = S.run_study(40, 200, [0.1], [0], 60, ["DP", "MP b=1", "DST d=1"], folds=10, emit=lines.append)
    assert len(rows) == 3 and len(lines) == 3
    by = {r["method"]: r for r in rows}
    for r in rows:
        assert "theta_hat" in r and r["evals"] <= 60 and r["iterations"] >= 1 and r["cv_folds"] == 10
        assert r["mspe"] is not None and r["mspe"] > 0
        json.loads(lines[rows.index(r)])
    dp, mp, dst = by["DP"], by["MP b=1"], by["DST d=1"]
    rel = max(abs(u - v) / abs(v) for u, v in zip(mp["theta_hat"], dp["theta_hat"]))
    assert rel <= 1e-3, (mp["theta_hat"], dp["theta_hat"])
    assert abs(mp["mspe"] - dp["mspe"]) <= 0.01 * dp["mspe"]
    assert dst["mspe"] >= 0.999 * dp["mspe"]
    summ = S.summary(rows, [0.1], ["DP", "MP b=1", "DST d=1"])
    assert {s["method"] for s in summ} == {"DP", "MP b=1", "DST d=1"}
    assert np.isclose(next(s for s in summ if s["method"] == "DP")["mean_mspe_ratio_to_dp"], 1.0)
    # resuming with every row done computes nothing and returns the same rows
    again = []
    rows2 = S.run_study(40, 200, [0.1], [0], 60, ["DP", "MP b=1", "DST d=1"], folds=10, emit=again.append,
                        done=rows)
    assert again == [] and rows2 == rows

"""Host logic of the search-form cost model (no GPU): the guided-search
replay, the training set built from measured records, and the measured
GB300 sweep shipped with the package -- its records are well formed and its
stored held-out evaluation is reproduced from the shipped parameters by the
FP64 oracle's forward pass."""
import json
import math

import numpy as np
import pytest

from oracle import costmodel as ocm
from paper_2311_04517_gb300 import costmodel as cm


def test_guided_choice_times_within_margin_only():
    ms = [1.0, 0.8, 2.0]
    sup = [1, 1, 1]
    # form 1 predicted fastest, form 0 within 25%, form 2 far off
    pred = [math.log(1.1), math.log(1.0), math.log(3.0)]
    assert cm.guided_choice(pred, ms, sup, 0.25) == (1, 2)
    # margin 0: only the best-ranked form is timed
    assert cm.guided_choice(pred, ms, sup, 0.0) == (1, 1)
    # a wrong ranking inside the margin is corrected by the timing
    pred = [math.log(1.0), math.log(1.2), math.log(3.0)]
    assert cm.guided_choice(pred, ms, sup, 0.25) == (1, 2)
    # unbuilt forms are never timed; equal predictions are within any margin
    assert cm.guided_choice([0.0, 0.0, 0.0], ms, [1, 0, 1], 0.0) == (0, 2)
    assert cm.guided_choice([0.0, -1.0, 0.0], ms, [1, 0, 1], 0.0) == (0, 2)
    # a huge margin times every built form
    assert cm.guided_choice(pred, ms, sup, 1e30) == (1, 3)


def test_library_plan():
    """hpc_costmodel_plan (host code of the library, no GPU): ranking by
    predicted time with ties to the lower form, unbuilt forms left out, the
    margin rule, and refusals."""
    from paper_2311_04517_gb300 import hpclust as H
    lg = math.log
    order, timed = H.hpc_costmodel_plan([lg(1.1), lg(1.0), lg(3.0)], [1, 1, 1], 0.25)
    assert order == [1, 0, 2] and timed == [1, 1, 0]
    order, timed = H.hpc_costmodel_plan([lg(1.1), lg(1.0), lg(3.0)], [1, 1, 1], 0.0)
    assert order == [1, 0, 2] and timed == [1, 0, 0]
    order, timed = H.hpc_costmodel_plan([0.0, 0.0, 0.0], [1, 0, 1], 0.0)
    assert order == [0, 2, -1] and timed == [1, 1, 0]
    order, timed = H.hpc_costmodel_plan([5.0, float("nan"), 1.0], [1, 0, 1], 1e30)
    assert order == [2, 0, -1] and timed == [1, 1, 0]
    for bad in (([float("nan"), 0.0, 0.0], [1, 1, 1], 0.1), ([0.0] * 3, [1, 1, 1], -0.5),
                ([0.0] * 3, [1, 1, 1], float("nan")), ([float("inf"), 0.0, 0.0], [1, 0, 0], 0.1)):
        with pytest.raises(H.HPCError):
            H.hpc_costmodel_plan(*bad)


def test_evaluate_counts():
    recs = [{"ms": [1.0, 2.0, -1.0], "supported": [1, 1, 0], "builtin": 1},
            {"ms": [3.0, 1.0, 1.02], "supported": [1, 1, 1], "builtin": 2}]
    preds = [[0.0, 1.0, 0.0], [0.0, 0.1, 5.0]]
    ev = cm.evaluate(recs, preds, margin=0.25)
    # case 1: form 0 timed alone (form 1 predicted e^1 slower) -> fastest
    # case 2: forms 0 and 1 timed (1.105 <= 1.25) -> form 1, the fastest
    assert ev["cases"] == 2 and ev["guided_within_5pct"] == 1.0
    assert ev["guided_forms_timed"] == 1.5 and ev["exhaustive_forms_timed"] == 2.5
    # built-in: case 1 wrong (2.0 vs 1.0), case 2 within 5% (1.02 vs 1.0)
    assert ev["builtin_within_5pct"] == 0.5


def test_dataset_targets_are_log_ns_per_row():
    recs = [{"n": 1 << 20, "ms": [2.0, -1.0, 0.5], "supported": [1, 0, 1],
             "features": [[0.0] * 8, [1.0] * 8, [2.0] * 8]}]
    X, t, where = cm.dataset(recs)
    assert X.shape == (2, 8) and where == [(0, 0), (0, 2)]
    assert t[0] == pytest.approx(math.log(2.0e6 / (1 << 20)), rel=1e-6)
    assert t[1] == pytest.approx(math.log(0.5e6 / (1 << 20)), rel=1e-6)
    assert np.all(X[1] == 2.0)


def test_init_params_layout():
    p = cm.init_params(0, 1.5)
    assert p.size == ocm.P and p.dtype == np.float32
    W1, b1, W2, b2, w3, b3 = ocm.unpack(p.astype(np.float64))
    assert np.all(b1 == 0) and np.all(b2 == 0) and b3 == 1.5
    assert 0.3 < np.std(W1) < 0.7 and 0.15 < np.std(W2) < 0.35


@pytest.mark.skipif(not cm.OUT.exists(), reason="no measured sweep shipped")
def test_shipped_sweep_and_its_evaluation():
    data = json.loads(cm.OUT.read_text())
    recs = data["records"]
    assert len(data["params"]) == ocm.P and data["device"].startswith("NVIDIA")
    for r in recs:
        assert sum(r["supported"]) >= 2
        for f in range(3):
            row = r["features"][f]
            assert row[4:7] == [1.0 if q == f else 0.0 for q in range(3)]
            assert row[0] == pytest.approx(math.log2(r["d"]) / 7, rel=1e-6)
            assert (r["ms"][f] > 0) == bool(r["supported"][f])
        assert r["supported"][r["builtin"]]
    train, held = cm.split(recs)
    assert {r["k"] for r in held} == set(cm.HOLDOUT_K)
    assert not {r["k"] for r in train} & set(cm.HOLDOUT_K)
    p = np.asarray(data["params"], dtype=np.float64)
    preds = [ocm.predict(p, np.asarray(r["features"])).tolist() for r in held]
    ev = cm.evaluate(held, preds)
    for key in ("cases", "guided_within_5pct", "guided_forms_timed", "builtin_within_5pct",
                "exhaustive_forms_timed"):
        assert ev[key] == pytest.approx(data["heldout"][key], abs=1.0 / len(held)), key
    # what the network gains: fewer forms timed than the exhaustive search,
    # and more often within 5% of the fastest than the built-in table
    assert ev["guided_forms_timed"] < ev["exhaustive_forms_timed"]
    assert ev["guided_within_5pct"] >= ev["builtin_within_5pct"]
    # training set: the stored loss fell by more than 100x
    assert data["train"]["loss_last"] < 0.01 * data["train"]["loss_first"]

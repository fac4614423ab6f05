"""What the trained predictor gains (CPU, no GPU needed): the packaged
network's most likely parameters, judged on held-out timing records.

The records (``paper_2306_10016_gb300/data/mlp_records_gb300.json.gz``,
written on a GB300 by ``python -m paper_2306_10016_gb300.predictor
--records``) hold, for ten problems larger than any training problem (2-D
rectangles up to 4096 x 2048, 3-D cubes up to 256^3, FP64), the grid
search's time and the device time of every combination of per-axis choices
the network can make, each a median of CUDA-graph replays with L2 evicted.
Here the network is evaluated by the FP64 oracle (O7) on the host, its top
valid class decoded per axis as HDC_PREDICT_MLP does, and its regret
T(choice) / T(grid search) - 1 read from the table, beside the two rules
without a network: explicit padding (q = 1 per axis) and q = 2 per axis."""
import gzip
import json
import os

import numpy as np
import pytest

import oracle
import paper_2306_10016_gb300 as hdc
from paper_2306_10016_gb300 import predictor

RECORDS = os.path.join(os.path.dirname(hdc.MLP_WEIGHTS), "mlp_records_gb300.json.gz")


def _load_checkpoint(path):
    with open(path, "rb") as fh:
        hdr = np.frombuffer(fh.read(20), dtype=np.int32)
        fh.read(8)  # step
        n_in, hid, n_out, npar = (int(x) for x in hdr[1:5])
        params = np.frombuffer(fh.read(4 * npar), dtype=np.float32)
    assert hdr[0] == 0x48444D4C
    return n_in, hid, n_out, params


@pytest.fixture(scope="module")
def packaged():
    if not (os.path.exists(hdc.MLP_WEIGHTS) and os.path.exists(RECORDS)):
        pytest.skip("no trained predictor or timing records in the package")
    hdc.build()
    n_in, hid, n_out, params = _load_checkpoint(hdc.MLP_WEIGHTS)
    assert (n_in, hid, n_out) == (hdc.MLP_FEATURES, hdc.MLP_HIDDEN, len(hdc.mlp_q_classes()) + 2)
    with gzip.open(RECORDS, "rt") as fh:
        recs = json.load(fh)
    p64 = params.astype(np.float64)

    def logits(X):
        n = X.shape[0]
        _, _, lg = oracle.mlp_loss_grad(p64, n_in, hid, n_out, X.astype(np.float64), np.zeros(n, np.int32),
                                        np.zeros(n, np.int32), n_out - 2)
        return lg

    return recs, logits


def test_network_choice_is_the_recorded_one(packaged):
    recs, logits = packaged
    for r in recs:
        prm = predictor.top_class_params(r["shape"], r["dtype"], logits)
        assert predictor.combo_key(prm) == r["network"], (r["shape"], prm)
        assert r["network"] in r["ms"]


def test_top_class_regret_within_ten_percent_and_beats_rules(packaged):
    recs, logits = packaged
    net = predictor.regret_table(recs, lambda r: predictor.combo_key(
        predictor.top_class_params(r["shape"], r["dtype"], logits)))
    explicit = predictor.regret_table(recs, lambda r: r["explicit"])
    q2 = predictor.regret_table(recs, lambda r: r["q2"])
    assert net["missing"] == 0
    assert net["geomean"] <= 0.10, net
    assert net["max"] <= 0.20, net
    assert net["geomean"] < explicit["geomean"], (net, explicit)
    assert net["geomean"] < q2["geomean"], (net, q2)


def test_records_cover_the_evaluation_problems(packaged):
    recs, _ = packaged
    assert [tuple(r["shape"]) for r in recs] == [tuple(s) for s in predictor.EVAL_PROBLEMS]
    train = set(predictor.training_problems(predictor.TRAIN_SEED, predictor.TRAIN_RECTANGLES))
    for r in recs:
        # held out: no evaluation problem is a training problem
        assert tuple(r["shape"]) not in train
        assert r["search_ms"] > 0 and all(v > 0 for v in r["ms"].values())
        # the grid search's own choice is in the table
        assert r["ms"][predictor.combo_key(r["search"])] == r["search_ms"]

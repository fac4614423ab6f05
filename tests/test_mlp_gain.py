"""What the trained predictor adds (CPU): on the grid-search dataset it was
trained on, the committed network (evaluated by the FP64 oracle, O7)
classifies the residue count far better than the best predictor-free
constant choice.  Regret on larger problems is measured on the GPU by
``python -m paper_2306_10016_gb300.predictor --eval``."""
import gzip
import json
import os

import numpy as np
import pytest

import oracle
import paper_2306_10016_gb300 as hdc
from paper_2306_10016_gb300 import predictor


def _load_checkpoint(path):
    with open(path, "rb") as fh:
        hdr = np.frombuffer(fh.read(20), dtype=np.int32)
        fh.read(8)  # step
        n_in, hid, n_out, npar = (int(x) for x in hdr[1:5])
        params = np.frombuffer(fh.read(4 * npar), dtype=np.float32)
    assert hdr[0] == 0x48444D4C
    return n_in, hid, n_out, params


@pytest.mark.skipif(not os.path.exists(hdc.MLP_WEIGHTS), reason="no trained predictor in the package")
def test_trained_predictor_beats_constant_rule():
    hdc.build()
    n_in, hid, n_out, params = _load_checkpoint(hdc.MLP_WEIGHTS)
    assert (n_in, hid, n_out) == (hdc.MLP_FEATURES, hdc.MLP_HIDDEN, len(hdc.mlp_q_classes()) + 2)
    with gzip.open(hdc.MLP_DATASET, "rt") as fh:
        recs = json.load(fh)
    X, yq, yd = predictor.samples(recs)
    _, _, logits = oracle.mlp_loss_grad(params.astype(np.float64), n_in, hid, n_out, X.astype(np.float64), yq, yd,
                                        n_out - 2)
    acc = float(np.mean(np.argmax(logits[:, :n_out - 2], axis=1) == yq))
    majority = float(np.bincount(yq).max() / yq.size)
    assert acc >= majority + 0.15, (acc, majority)
    # the decoded parameters are valid tuples for every sample
    for r in recs[:50]:
        for a, L in enumerate(r["L"]):
            prm = hdc.mlp_decode_axis(np.zeros(n_out, dtype=np.float32), L, 2 * L - 1)
            assert prm["q"] * prm["m"] >= 2 * L - 1

"""Pins for the predictor network's FP64 oracle (O7): gradients against
central finite differences of its own loss, the loss against a numpy
forward pass, Adam against its published update written out in numpy."""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth

N_IN, H, N_Q = 5, 7, 4
N_OUT = N_Q + 2


def _setup(seed=3, n=6):
    npar = oracle.mlp_num_params(N_IN, H, N_OUT)
    P = 0.5 * (2 * synth.uniform01(seed, npar) - 1)
    X = 2 * synth.uniform01(seed + 1, n * N_IN).reshape(n, N_IN) - 1
    yq = np.array([0, 3, 1, -1, 2, 2][:n], dtype=np.int32)
    yd = np.array([1, 0, -1, 1, 0, 1][:n], dtype=np.int32)
    return P, X, yq, yd


def _numpy_loss(P, X, yq, yd):
    dims = [N_IN, H, H, H, N_OUT]
    off = 0
    a = X
    for l in range(4):
        W = P[off:off + dims[l] * dims[l + 1]].reshape(dims[l], dims[l + 1])
        off += dims[l] * dims[l + 1]
        b = P[off:off + dims[l + 1]]
        off += dims[l + 1]
        a = a @ W + b
        if l < 3:
            a = np.maximum(a, 0)
    tot = 0.0
    for s in range(X.shape[0]):
        for lo, hi, y in ((0, N_Q, yq[s]), (N_Q, N_Q + 2, yd[s])):
            if y < 0:
                continue
            z = a[s, lo:hi]
            tot += np.log(np.sum(np.exp(z - z.max()))) + z.max() - z[y]
    return tot / X.shape[0], a


def test_loss_and_logits_match_numpy():
    P, X, yq, yd = _setup()
    loss, _, logits = oracle.mlp_loss_grad(P, N_IN, H, N_OUT, X, yq, yd, N_Q)
    ref_loss, ref_logits = _numpy_loss(P, X, yq, yd)
    assert abs(loss - ref_loss) < 1e-12
    assert np.max(np.abs(logits - ref_logits)) < 1e-12


def test_gradient_matches_finite_differences():
    P, X, yq, yd = _setup(seed=9)
    _, grad, _ = oracle.mlp_loss_grad(P, N_IN, H, N_OUT, X, yq, yd, N_Q)
    eps = 1e-6
    rng = np.random.default_rng(0)
    idx = np.unique(np.concatenate([np.arange(0, P.size, 7), rng.integers(0, P.size, 40)]))
    for k in idx:
        Pp = P.copy(); Pp[k] += eps
        Pm = P.copy(); Pm[k] -= eps
        lp = oracle.mlp_loss_grad(Pp, N_IN, H, N_OUT, X, yq, yd, N_Q)[0]
        lm = oracle.mlp_loss_grad(Pm, N_IN, H, N_OUT, X, yq, yd, N_Q)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grad[k]) < 1e-6 * max(1.0, abs(fd)), k


def test_adam_matches_written_out_update():
    rng = np.random.default_rng(1)
    p = rng.standard_normal(20)
    m = np.zeros(20)
    v = np.zeros(20)
    p_ref, m_ref, v_ref = p.copy(), m.copy(), v.copy()
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    for t in range(1, 4):
        g = rng.standard_normal(20)
        oracle.adam_step(p, g, m, v, lr, b1, b2, eps, t)
        m_ref = b1 * m_ref + (1 - b1) * g
        v_ref = b2 * v_ref + (1 - b2) * g * g
        p_ref = p_ref - lr * (m_ref / (1 - b1 ** t)) / (np.sqrt(v_ref / (1 - b2 ** t)) + eps)
    assert np.max(np.abs(p - p_ref)) < 1e-14

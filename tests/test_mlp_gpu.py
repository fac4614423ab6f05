"""The predictor network's CUDA kernels against the FP64 oracle (O7):
forward logits, loss, gradients, Adam; training, checkpoint resume and
prediction through plans."""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_10016_gb300 as h
    h.build()
    h.lib()
    return h


def _data(n, n_in, nq, seed):
    X = (2 * synth.uniform01(seed, n * n_in) - 1).reshape(n, n_in).astype(np.float32)
    u = synth.uniform01(seed + 1, 2 * n)
    yq = (u[:n] * nq).astype(np.int32)
    yd = (u[n:] * 2).astype(np.int32)
    yq[::7] = -1
    yd[::5] = -1
    return X, yq, yd


def test_forward_loss_grad_vs_oracle(hdc):
    from paper_2306_10016_gb300.predictor import init_params
    net = hdc.MLP()
    nq = net.n_out - 2
    P = init_params(net.n_in, net.hidden, net.n_out, 77)
    net.set_params(P)
    X, yq, yd = _data(37, net.n_in, nq, 5)
    Xd = torch.from_numpy(X).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.loss_grad(Xd, torch.from_numpy(yq).cuda(), torch.from_numpy(yd).cuda(), loss)
    logits = net.forward(Xd).cpu().numpy()
    torch.cuda.synchronize()
    l_ref, g_ref, lg_ref = oracle.mlp_loss_grad(P.astype(np.float64), net.n_in, net.hidden, net.n_out,
                                                X.astype(np.float64), yq, yd, nq)
    assert rel_max_err(logits, lg_ref) < 1e-5
    assert abs(float(loss.item()) - l_ref) < 1e-5 * max(1.0, abs(l_ref))
    assert rel_max_err(net.grads(), g_ref) < 1e-4


def test_adam_step_vs_oracle(hdc):
    from paper_2306_10016_gb300.predictor import init_params
    net = hdc.MLP()
    nq = net.n_out - 2
    P = init_params(net.n_in, net.hidden, net.n_out, 78)
    net.set_params(P)
    X, yq, yd = _data(16, net.n_in, nq, 6)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    p = P.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(1, 4):
        net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(yq).cuda(), torch.from_numpy(yd).cuda(), loss)
        g = net.grads().astype(np.float64)
        net.adam(1e-2)
        torch.cuda.synchronize()
        p_gpu_before = p.copy()
        oracle.adam_step(p, g, m, v, 1e-2, 0.9, 0.999, 1e-8, t)
        got = net.params().astype(np.float64)
        assert np.max(np.abs(got - p)) < 1e-5, t
        p = got  # continue from the GPU's own float32 parameters
        _ = p_gpu_before


def test_training_learns_a_separable_rule(hdc):
    from paper_2306_10016_gb300.predictor import accuracy, train
    n, nq, F = 400, 8, hdc.MLP_FEATURES
    X = (2 * synth.uniform01(11, n * F) - 1).reshape(n, F).astype(np.float32)
    yq = np.clip(((X[:, 0] + 1) * 4).astype(np.int32), 0, nq - 1)   # class from the first feature
    yd = (X[:, 1] > 0).astype(np.int32)
    net, hist = train(X, yq, yd, steps=600, lr=1e-2)
    assert hist[-1][1] < 0.5 * hist[0][1]
    aq, ad = accuracy(net, X, yq, yd)
    assert aq > 0.85 and ad > 0.9


def test_checkpoint_resume_is_exact(hdc, tmp_path):
    from paper_2306_10016_gb300.predictor import init_params
    X, yq, yd = _data(32, hdc.MLP_FEATURES, 8, 12)
    Xd, yqd, ydd = torch.from_numpy(X).cuda(), torch.from_numpy(yq).cuda(), torch.from_numpy(yd).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def steps(net, k):
        for _ in range(k):
            net.loss_grad(Xd, yqd, ydd, loss)
            net.adam(5e-3)
        torch.cuda.synchronize()

    a = hdc.MLP()
    a.set_params(init_params(hdc.MLP_FEATURES, 64, a.n_out, 3))
    steps(a, 10)
    a.save(tmp_path / "ck.bin")
    steps(a, 10)
    b = hdc.MLP()
    b.load(tmp_path / "ck.bin")
    steps(b, 10)
    assert np.array_equal(a.params(), b.params())


def test_plan_predict_mlp(hdc, tmp_path):
    """A network trained to always answer q = 2, D = q drives a plan whose
    convolution is correct."""
    from paper_2306_10016_gb300.predictor import train
    F = hdc.MLP_FEATURES
    X = (2 * synth.uniform01(21, 200 * F) - 1).reshape(200, F).astype(np.float32)
    yq = np.full(200, hdc.mlp_q_to_class(2), dtype=np.int32)
    yd = np.zeros(200, dtype=np.int32)
    train(X, yq, yd, steps=200, lr=1e-2, checkpoint=str(tmp_path / "w.bin"))
    shape = (300, 200)
    pl = hdc.Plan(list(shape), mode=hdc.HDC_PREDICT_MLP, tuning_db=str(tmp_path / "w.bin"))
    for a, L in zip(pl.params, shape):
        assert a["q"] == 2 and a["m"] == hdc.next_good_size(-(-(2 * L - 1) // 2)) and a["D"] == 2
    f = synth.unit_disk(31, shape)
    g = synth.unit_disk(32, shape)
    h = pl.execute(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert rel_max_err(h.cpu().numpy(), oracle.conv_fft(f, g)) < 1e-12
    # a missing weights file is reported, not guessed around
    with pytest.raises(hdc.HDCError) as ei:
        hdc.Plan(list(shape), mode=hdc.HDC_PREDICT_MLP, tuning_db=str(tmp_path / "none.bin"))
    assert ei.value.code == hdc.HDC_ERR_NOT_TUNED


def test_plan_predict_mlp_search_packaged(hdc):
    """The packaged predictor with the guided search of its three best
    classes per axis gives a valid, correct plan."""
    import os
    if not os.path.exists(hdc.MLP_WEIGHTS):
        pytest.skip("no trained predictor in the package")
    shape = (96, 320)
    pl = hdc.Plan(list(shape), mode=hdc.HDC_PREDICT_MLP_SEARCH)
    prm = pl.params
    assert all(p["q"] * p["m"] >= 2 * L - 1 for p, L in zip(prm, shape))
    f = synth.unit_disk(41, shape)
    g = synth.unit_disk(42, shape)
    h = pl.execute(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    assert rel_max_err(h.cpu().numpy(), oracle.conv_fft(f, g)) < 1e-12


def test_guided_search_candidates_and_decode_class(hdc):
    """The packaged guided search times at most six candidates per axis, and
    decoding a class index agrees with decoding the top-ranked logits."""
    import numpy as np
    pl = hdc.Plan([1024, 384], mode=hdc.HDC_PREDICT_MLP_SEARCH)
    assert 2 <= pl.timed <= 12
    assert hdc.Plan([1024, 384], mode=hdc.HDC_PREDICT_MLP).timed == 0
    nq = hdc.mlp_num_q_classes() if hasattr(hdc, "mlp_num_q_classes") else 8
    for k in range(nq):
        lg = np.full(nq + 2, -5.0, dtype=np.float32)
        lg[k] = 5.0
        lg[nq] = 1.0                       # D head: D = q
        try:
            want = hdc.mlp_decode_axis(lg, 3000, 5999, hdc.HDC_C128)
        except hdc.HDCError:
            continue
        m, p, q, D = (hdc.C.c_int64() for _ in range(4))
        rc = hdc.lib().hdc_mlp_decode_class(k, 0, 3000, 5999, hdc.HDC_C128, 0, hdc.C.byref(m), hdc.C.byref(p),
                                            hdc.C.byref(q), hdc.C.byref(D))
        if rc == 0 and want["m"] == m.value:
            assert (want["p"], want["q"], want["D"]) == (p.value, q.value, D.value)

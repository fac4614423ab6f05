"""Parity at the sizes the measured configurations run, element by element
against the CPU oracle (through the C ABI):

* 2-D 1024 x 1024 and 3-D 128^3 complex convolutions (M = 2L - 1 per axis)
  with the tuples the tuner picks for them and with explicit padding, FP64
  and FP32, against the explicitly padded FFT convolution (O2);
* the batched configuration: 4096 convolutions with L log-uniform in
  [64, 65536] (seed BASE_SEED + 4), per-size-class m from the batched
  tuner, one persistent launch: every convolution with L <= 4096 against the
  direct sum (O1), a seeded sample of the longer ones in full against O2;
* FP32 at the sweep sizes 2^17 .. 2^22 and 3 * 2^16 .. 3 * 2^20, in full
  against the closed form of exponential sequences (O4) and against O2 on
  unit-disk inputs, for implicit (q = 2), hybrid (q = 4) and explicit
  (q = 1) tuples.

Tolerances: relative max-norm error <= 1e-12 (FP64) and <= 5e-5 (FP32)."""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 5e-5}


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_10016_gb300 as h
    h.build()
    h.lib()
    return h


ND_CASES = [
    # shape, m per axis, D per axis: the tuner's choices for these shapes
    # (one residue pair per pass in 2-D), explicit padding, and more passes
    ((1024, 1024), [1024, 1024], [2, 2]),
    ((1024, 1024), [2048, 2048], [1, 1]),
    ((1024, 1024), [1024, 1536], [1, 2]),
    ((128, 128, 128), [128, 128, 256], [2, 2, 1]),
    ((128, 128, 128), [256, 256, 256], [1, 1, 1]),
]


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("shape,m,D", ND_CASES)
def test_nd_config_sizes(hdc, dt, shape, m, D):
    f = synth.unit_disk(synth.BASE_SEED + 30, shape)
    g = synth.unit_disk(synth.BASE_SEED + 31, shape)
    ref = oracle.conv_fft(f, g)
    ft = torch.from_numpy(f).to("cuda", dt)
    gt = torch.from_numpy(g).to("cuda", dt)
    h = hdc.convnd(ft, gt, len(shape), m, D=D)
    torch.cuda.synchronize()
    err = rel_max_err(h.cpu().numpy().astype(np.complex128), ref)
    assert err <= TOL[dt], (shape, m, D, err)


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64])
def test_batched_config_size(hdc, dt):
    n = 4096
    Ls = [int(x) for x in synth.log_uniform_lengths(synth.BASE_SEED + 4, n, 64, 65536)]
    tot = sum(Ls)
    fa = synth.unit_disk(synth.BASE_SEED + 40, (tot,))
    ga = synth.unit_disk(synth.BASE_SEED + 41, (tot,))
    offs = np.concatenate([[0], np.cumsum(Ls)])
    ft = torch.from_numpy(fa).to("cuda", dt)
    gt = torch.from_numpy(ga).to("cuda", dt)
    ht = torch.full_like(ft, complex("nan+nanj"))
    fs = [ft[offs[i]:offs[i + 1]] for i in range(n)]
    gs = [gt[offs[i]:offs[i + 1]] for i in range(n)]
    hs = [ht[offs[i]:offs[i + 1]] for i in range(n)]
    ms, _ = hdc.batched_tune(fs, gs, hs, reps=1, max_cands=4)
    plan = hdc.BatchedPlan(Ls, ms, hdc.dtype_code(dt))
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.bind(fs, gs, hs)
    ht.fill_(complex("nan+nanj"))
    plan.execute(ws)
    torch.cuda.synchronize()
    assert hdc.BatchedPlan.status(ws) == 0
    out = ht.cpu().numpy().astype(np.complex128)
    short = [i for i in range(n) if Ls[i] <= 4096]
    long_ = [i for i in range(n) if Ls[i] > 4096]
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    sample = sorted(rng.choice(long_, size=min(48, len(long_)), replace=False).tolist())
    worst = 0.0
    for i in short + sample:
        f = fa[offs[i]:offs[i + 1]]
        g = ga[offs[i]:offs[i + 1]]
        ref = oracle.conv_direct(f, g) if Ls[i] <= 4096 else oracle.conv_fft(f, g)
        err = rel_max_err(out[offs[i]:offs[i + 1]], ref)
        worst = max(worst, err)
        assert err <= TOL[dt], (i, Ls[i], ms[i], err)
    assert len(short) > 2000 and worst > 0.0


SWEEP32 = [1 << k for k in range(17, 23)] + [3 << k for k in range(16, 21)]


@pytest.mark.parametrize("L", SWEEP32)
def test_fp32_sweep_sizes_in_full(hdc, L):
    M = 2 * L - 1
    # exponential sequences: the closed form of O4, every output
    A, B, P = 123457, 98765, (1 << 26) + 7
    fe = synth.exp_seq(A, P, L)
    ge = synth.exp_seq(B, P, L)
    ref_e = oracle.closed_form_exp(A, B, P, L)
    # unit-disk inputs: O2, every output
    fu = synth.unit_disk(synth.BASE_SEED + 10 + L % 97, (L,))
    gu = synth.unit_disk(synth.BASE_SEED + 1010 + L % 97, (L,))
    ref_u = oracle.conv_fft(fu, gu)
    tuples = [(L, 2), (hdc.next_good_size(-(-M // 4)), 4), (hdc.next_good_size(M), 1)]
    for m, q in tuples:
        for f, g, ref in ((fe, ge, ref_e), (fu, gu, ref_u)):
            ft = torch.from_numpy(f).to("cuda", torch.complex64)
            gt = torch.from_numpy(g).to("cuda", torch.complex64)
            h = hdc.conv1d(ft, gt, m)
            torch.cuda.synchronize()
            err = rel_max_err(h.cpu().numpy().astype(np.complex128), ref)
            assert err <= TOL[torch.complex64], (L, m, q, err)

"""Parity of the multi-convolution (the n-fold convolution of n arrays,
hdc_convnd_multi through the C ABI) with the CPU oracle.

References: O9 (residue transforms, all n inputs) on small cases; iterated
first-L convolutions by O1 (direct) or O2 (explicit FFT) on larger and
N-D cases (the first L outputs of an n-fold convolution depend only on the
first L outputs of every partial product); O1 at sampled outputs at full
size.  Tolerances: relative max-norm error <= 1e-12 in FP64, <= 5e-5 in FP32.
"""
from functools import reduce

import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err, check_best_timed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 5e-5


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_10016_gb300 as h
    h.build()
    h.lib()
    return h


def dev(a, dtype=np.complex128):
    tdt = torch.complex128 if dtype == np.complex128 else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to("cuda", tdt)


def run(hdc, xs, dims, m, dtype=np.complex128, **kw):
    h = hdc.convnd_multi([dev(x, dtype) for x in xs], dims, m, **kw)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.complex128)


def iterated(xs, method="direct"):
    fn = oracle.conv_direct if method == "direct" else oracle.conv_fft
    return reduce(fn, [np.asarray(x) for x in xs])


def good(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def test_grid_small_against_o9(hdc):
    cnt = 0
    for n in (2, 3, 4, 8):
        for L in (1, 5, 17, 40):
            xs = synth.unit_disk(1000 + 10 * n + L, (n, 2, L))
            M = n * (L - 1) + 1
            for m in [k for k in range(1, 2 * M + 2) if good(k)][:: max(1, M // 12)]:
                q = -(-M // m)
                for D in sorted({1, q}):
                    h = run(hdc, xs, 1, m, D=D)
                    for b in range(2):
                        ref = oracle.conv_multi(xs[:, b, :], m)
                        assert rel_max_err(h[b], ref) < TOL64, (n, L, m, D)
                    cnt += 1
    assert cnt > 80


def test_two_inputs_match_convnd_bitwise(hdc):
    L = 3000
    f = synth.unit_disk(1101, (2, L))
    g = synth.unit_disk(1102, (2, L))
    for m, D in ((1024, 1), (6000, 0), (8192, 0)):
        a = run(hdc, [f, g], 1, m, D=D)
        b = hdc.convnd(dev(f), dev(g), 1, m, D=D).cpu().numpy()
        assert np.array_equal(a, b), (m, D)


def test_split_route_and_passes(hdc):
    L = 20000
    xs = synth.unit_disk(1201, (3, L))
    ref = iterated(xs, "fft")
    for m, D in ((8192, 0), (8192, 2), (65536, 0), (1000, 3), (2048, 0)):
        h = run(hdc, xs, 1, m, D=D)
        assert rel_max_err(h, ref) < TOL64, (m, D)
    xs = synth.unit_disk(1202, (5, 4, 3000))
    ref = np.stack([iterated(xs[:, b], "fft") for b in range(4)])
    h = run(hdc, xs, 1, 4096)
    assert rel_max_err(h, ref) < TOL64


def test_exact_integers(hdc):
    n, L = 4, 1000
    parts = [synth.small_ints(1300 + i, (L,)) for i in range(n)]
    re, im = parts[0]
    for re2, im2 in parts[1:]:
        re, im = oracle.conv_int_exact(re, im, re2, im2)
    xs = [r + 1j * i for r, i in parts]
    for m in (512, 4000, 1024):
        h = run(hdc, xs, 1, m)
        assert np.array_equal(np.rint(h.real).astype(np.int64), re), m
        assert np.array_equal(np.rint(h.imag).astype(np.int64), im), m


def test_fp32(hdc):
    xs = synth.unit_disk(1401, (3, 2, 5000))
    ref = np.stack([iterated(xs[:, b], "fft") for b in range(2)])
    for m in (1024, 16384):
        h = run(hdc, xs, 1, m, dtype=np.complex64)
        assert rel_max_err(h, ref) < TOL32, m


def test_full_size_sampled(hdc):
    """n = 3 inputs of 2^20 points; sampled outputs against O1 applied to
    the oracle's (O2) first-2^20 product of the first two inputs."""
    L = 1 << 20
    xs = synth.unit_disk(1501, (3, L))
    h = run(hdc, xs, 1, 1 << 20)
    u = oracle.conv_fft(xs[0], xs[1])
    rng = np.random.default_rng(3)
    idx = np.concatenate([[0, 1, L - 1], rng.integers(0, L, 45)]).astype(np.int64)
    ref = oracle.conv_direct_at(u, xs[2], idx)
    assert rel_max_err(h[idx], ref) < TOL64


def test_2d_and_3d(hdc):
    xs = synth.unit_disk(1601, (3, 2, 20, 24))
    ref = np.stack([iterated(xs[:, b]) for b in range(2)])
    for m, D in (((16, 32), (0, 0)), ((64, 8), (1, 2)), ((9, 70), (0, 1))):
        h = run(hdc, xs, 2, list(m), D=list(D))
        assert rel_max_err(h, ref) < TOL64, (m, D)
    xs = synth.unit_disk(1602, (4, 6, 7, 8))
    ref = iterated(xs)
    for m in ((8, 8, 8), (21, 25, 29), (32, 32, 32)):
        if not all(good(v) for v in m):
            continue
        h = run(hdc, xs, 3, list(m))
        assert rel_max_err(h, ref) < TOL64, m


def test_errors(hdc):
    xs = [dev(synth.unit_disk(1700 + i, (30,))) for i in range(3)]
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_multi(xs, 1, 64, M=59)              # 2 L - 1: enough for two inputs only
    assert e.value.code == hdc.HDC_ERR_ALIAS
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_multi(xs, 1, 64, out=xs[1])
    assert e.value.code == hdc.HDC_ERR_PARAM
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_multi(xs * 3, 1, 512)               # nine inputs
    assert e.value.code == hdc.HDC_ERR_PARAM


def test_tuner(hdc):
    xs = [dev(synth.unit_disk(1800 + i, (2, 3000))) for i in range(3)]
    best, trials = hdc.tune_multi(xs, 1, reps=2)
    assert trials
    check_best_timed(best, trials)
    h = hdc.convnd_multi(xs, 1, best[0]["m"], D=best[0]["D"]).cpu().numpy()
    ref = np.stack([iterated([x.cpu().numpy()[b] for x in xs], "fft") for b in range(2)])
    assert rel_max_err(h, ref) < TOL64


# ------------------------------------------------- sum of pairwise products

def pairwise(xs, method="direct"):
    fn = oracle.conv_direct if method == "direct" else oracle.conv_fft
    return sum(fn(np.asarray(xs[i]), np.asarray(xs[i + 1])) for i in range(0, len(xs), 2))


def test_dot_grid_small_against_o9(hdc):
    cnt = 0
    for n in (2, 4, 8):
        for L in (1, 6, 23):
            xs = synth.unit_disk(1900 + 10 * n + L, (n, 2, L))
            M = 2 * L - 1
            for m in [k for k in range(1, 2 * M + 2) if good(k)][:: max(1, M // 8)]:
                q = -(-M // m)
                for D in sorted({1, q}):
                    h = run(hdc, xs, 1, m, op="dot", D=D)
                    for b in range(2):
                        ref = oracle.conv_multi(xs[:, b, :], m, op="dot")
                        assert rel_max_err(h[b], ref) < TOL64, (n, L, m, D)
                    cnt += 1
    assert cnt > 30


def test_dot_routes_nd_and_integers(hdc):
    xs = synth.unit_disk(2001, (4, 3, 20000))
    ref = np.stack([pairwise(xs[:, b], "fft") for b in range(3)])
    for m, D in ((40000, 0), (65536, 0), (1250, 4), (2048, 0)):
        h = run(hdc, xs, 1, m, op="dot", D=D)
        assert rel_max_err(h, ref) < TOL64, (m, D)
    xs = synth.unit_disk(2002, (6, 20, 24))
    h = run(hdc, xs, 2, [40, 48], op="dot")
    assert rel_max_err(h, pairwise(xs)) < TOL64
    xs = synth.unit_disk(2003, (4, 5, 6, 7))
    h = run(hdc, xs, 3, [9, 12, 14], op="dot")
    assert rel_max_err(h, pairwise(xs)) < TOL64
    parts = [synth.small_ints(2100 + i, (2000,)) for i in range(8)]
    re = np.zeros(2000, dtype=np.int64)
    im = np.zeros(2000, dtype=np.int64)
    for i in range(0, 8, 2):
        a, b = oracle.conv_int_exact(*parts[i], *parts[i + 1])
        re += a
        im += b
    h = run(hdc, [r + 1j * i for r, i in parts], 1, 4000, op="dot")
    assert np.array_equal(np.rint(h.real).astype(np.int64), re)
    assert np.array_equal(np.rint(h.imag).astype(np.int64), im)
    h = run(hdc, [r + 1j * i for r, i in parts], 1, 4000, op="dot", dtype=np.complex64)
    assert rel_max_err(h, re + 1j * im) < TOL32


def test_dot_two_inputs_match_convnd_bitwise_and_errors(hdc):
    f = synth.unit_disk(2201, (2, 3000))
    g = synth.unit_disk(2202, (2, 3000))
    a = run(hdc, [f, g], 1, 6000, op="dot")
    b = hdc.convnd(dev(f), dev(g), 1, 6000).cpu().numpy()
    assert np.array_equal(a, b)
    xs = [dev(synth.unit_disk(2300 + i, (30,))) for i in range(3)]
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_multi(xs, 1, 64, op="dot")           # odd number of inputs
    assert e.value.code == hdc.HDC_ERR_PARAM
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_multi(xs[:2] * 2, 1, 64, op="dot", M=58)
    assert e.value.code == hdc.HDC_ERR_ALIAS

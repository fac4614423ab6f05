"""Parity of the real-input convolution (hdc_convnd_real: packed f + i g,
conjugate residue pairs) with the CPU oracle.

References: O10 on small 1-D cases; O1/O2 on the inputs as complex arrays
(real part) for larger and N-D cases; exact integers (O3).  Tolerances:
relative max-norm error <= 1e-12 in FP64, <= 5e-5 in FP32.
"""
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


def real_pair(seed, shape):
    z = synth.unit_disk(seed, shape)
    return np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)


def run(hdc, f, g, dims, m, dtype=np.float64, **kw):
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    ft = torch.from_numpy(np.ascontiguousarray(f, dtype=dtype)).to("cuda", tdt)
    gt = torch.from_numpy(np.ascontiguousarray(g, dtype=dtype)).to("cuda", tdt)
    h = hdc.convnd_real(ft, gt, dims, m, **kw)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.float64)


def good(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def cref(f, g, method="direct"):
    fn = oracle.conv_direct if method == "direct" else oracle.conv_fft
    return fn(np.asarray(f, dtype=complex), np.asarray(g, dtype=complex)).real


def test_grid_small_against_o10(hdc):
    n = 0
    for L in (1, 2, 5, 12, 33):
        f, g = real_pair(100 + L, (2, L))
        M = 2 * L - 1
        for m in [k for k in range(1, 2 * M + 2) if good(k)]:
            q = -(-M // m)
            for D in sorted({1, q // 2 + 1}):
                h = run(hdc, f, g, 1, m, D=D)
                for b in range(2):
                    assert rel_max_err(h[b], oracle.conv_real(f[b], g[b], m)) < TOL64, (L, m, D)
                n += 1
    assert n > 60


def test_routes_passes_and_batch(hdc):
    f, g = real_pair(201, (3, 20000))
    ref = np.stack([cref(f[b], g[b], "fft") for b in range(3)])
    for m, D in ((40000, 0), (65536, 0), (8192, 1), (8192, 0), (2048, 3), (1250, 0), (5000, 2)):
        h = run(hdc, f, g, 1, m, D=D)
        assert rel_max_err(h, ref) < TOL64, (m, D)


def test_exact_integers_and_fp32(hdc):
    L = 3000
    fi, _ = synth.small_ints(301, (L,))
    gi, _ = synth.small_ints(302, (L,))
    zero = np.zeros(L, dtype=np.int64)
    hre, _ = oracle.conv_int_exact(fi, zero, gi, zero)
    for m in (6000, 1024, 8192):
        h = run(hdc, fi.astype(float), gi.astype(float), 1, m)
        assert np.array_equal(np.rint(h).astype(np.int64), hre), m
    f, g = real_pair(303, (2, 5000))
    ref = np.stack([cref(f[b], g[b], "fft") for b in range(2)])
    for m in (1024, 10000, 16384):
        h = run(hdc, f, g, 1, m, dtype=np.float32)
        assert rel_max_err(h, ref) < TOL32, m


def test_full_size_sampled(hdc):
    L = 1 << 22
    f, g = real_pair(401, (L,))
    h = run(hdc, f, g, 1, 1 << 22)
    rng = np.random.default_rng(5)
    idx = np.concatenate([[0, 1, L - 1], rng.integers(0, L, 45)]).astype(np.int64)
    ref = oracle.conv_direct_at(f.astype(complex), g.astype(complex), idx).real
    assert rel_max_err(h[idx], ref) < TOL64


def test_2d_3d(hdc):
    f, g = real_pair(501, (2, 20, 24))
    ref = np.stack([cref(f[b], g[b]) for b in range(2)])
    for m, D in (((40, 48), (0, 0)), ((16, 16), (1, 2)), ((9, 70), (2, 0)), ((64, 8), (0, 0))):
        h = run(hdc, f, g, 2, list(m), D=list(D))
        assert rel_max_err(h, ref) < TOL64, (m, D)
    f, g = real_pair(502, (6, 7, 8))
    ref = cref(f, g)
    for m in ((12, 14, 16), (4, 7, 8), (16, 16, 16)):
        h = run(hdc, f, g, 3, list(m))
        assert rel_max_err(h, ref) < TOL64, m
    f, g = real_pair(503, (64, 3000))
    ref = cref(f, g, "fft")
    h = run(hdc, f, g, 2, [128, 8192])
    assert rel_max_err(h, ref) < TOL64


def test_matches_complex_path(hdc):
    """The real path and the complex path on the same inputs (imaginary parts
    zero) agree to rounding."""
    f, g = real_pair(601, (4, 6000))
    hr = run(hdc, f, g, 1, 4096)
    hc = hdc.convnd(torch.from_numpy(f.astype(complex)).cuda(), torch.from_numpy(g.astype(complex)).cuda(), 1,
                    4096).cpu().numpy()
    assert np.max(np.abs(hc.imag)) < 1e-12 * np.max(np.abs(hc.real))
    assert rel_max_err(hr, hc.real) < TOL64


def test_errors(hdc):
    f = torch.zeros(30, dtype=torch.float64, device="cuda")
    g = torch.zeros(30, dtype=torch.float64, device="cuda")
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_real(f, g, 1, 16, M=58)
    assert e.value.code == hdc.HDC_ERR_ALIAS
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_real(f, g, 1, 16, out=f)
    assert e.value.code == hdc.HDC_ERR_PARAM
    with pytest.raises(TypeError):
        hdc.convnd_real(f.to(torch.complex128), g.to(torch.complex128), 1, 16)


def test_tuner(hdc):
    f, g = real_pair(701, (2, 5000))
    ft = torch.from_numpy(f).cuda()
    gt = torch.from_numpy(g).cuda()
    best, trials = hdc.tune_real(ft, gt, 1, reps=2)
    assert trials
    check_best_timed(best, trials)
    h = run(hdc, f, g, 1, best[0]["m"], D=best[0]["D"])
    ref = np.stack([cref(f[b], g[b], "fft") for b in range(2)])
    assert rel_max_err(h, ref) < TOL64

"""Parity of the unequal-length convolution (Section 3.5 residue matching,
hdc_convnd_unequal through the C ABI) with the CPU oracle.

References: O8 (the paper's unequal algorithm, 1-D) on small cases; the
oracle's explicit FFT convolution (O2) or direct sums (O1) of the inputs
zero-padded to the length of the linear convolution on larger and N-D
cases; O1 at sampled outputs at full size.  Tolerances: relative max-norm
error <= 1e-12 in FP64, <= 5e-5 in FP32.
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


def dev(a, dtype=np.complex128):
    tdt = torch.complex128 if dtype == np.complex128 else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to("cuda", tdt)


def run(hdc, f, g, dims, m, lam=1, dtype=np.complex128, **kw):
    h = hdc.convnd_unequal(dev(f, dtype), dev(g, dtype), dims, m, lam, **kw)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.complex128)


def padded_full(f, g, dims):
    """f and g zero-padded to the shape of their full linear convolution
    over the last `dims` axes (leading axes kept)."""
    lead = f.shape[: f.ndim - dims]
    S = [a + b - 1 for a, b in zip(f.shape[f.ndim - dims:], g.shape[g.ndim - dims:])]
    fp = np.zeros(lead + tuple(S), dtype=complex)
    gp = np.zeros(lead + tuple(S), dtype=complex)
    fp[(...,) + tuple(slice(0, n) for n in f.shape[f.ndim - dims:])] = f
    gp[(...,) + tuple(slice(0, n) for n in g.shape[g.ndim - dims:])] = g
    return fp, gp


def full_conv(f, g, dims, method="direct"):
    fp, gp = padded_full(f, g, dims)
    fn = oracle.conv_direct if method == "direct" else oracle.conv_fft
    if fp.ndim == dims:
        return fn(fp, gp)
    return np.stack([fn(a, b) for a, b in zip(fp.reshape((-1,) + fp.shape[-dims:]),
                                              gp.reshape((-1,) + gp.shape[-dims:]))]).reshape(
        fp.shape[: fp.ndim - dims] + fp.shape[-dims:])


def good(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


# ------------------------------------------------------------------ 1-D

def test_grid_small_against_o8(hdc):
    """Every (m, lam) with m, lam m good, lam <= 5, on a few length pairs,
    D in {1, qg}, two batch rows; reference O8 per row."""
    n = 0
    for Lf, Lg in ((1, 9), (3, 20), (17, 20), (5, 64), (20, 7)):
        f = synth.unit_disk(100 + Lf, (2, Lf))
        g = synth.unit_disk(200 + Lg, (2, Lg))
        for m in (1, 2, 3, 4, 5, 8, 16):
            for lam in (1, 2, 3, 4, 5):
                if not good(lam * m):
                    continue
                _, _, qg, _ = hdc.validate_unequal_axis(Lf, Lg, m, lam)
                for D in sorted({1, qg}):
                    h = run(hdc, f, g, 1, m, lam, D=D)
                    for b in range(2):
                        ref = oracle.conv_unequal(f[b], g[b], m, lam)
                        assert rel_max_err(h[b], ref) < TOL64, (Lf, Lg, m, lam, D)
                    n += 1
    assert n > 100


def test_windows_and_padding(hdc):
    f = synth.unit_disk(11, (13,))
    g = synth.unit_disk(12, (31,))
    for m, lam, M, o, Lw in ((4, 3, None, 0, 43), (4, 3, 60, 10, 33), (8, 2, 48, 5, 20), (2, 8, None, 0, 31)):
        h = run(hdc, f, g, 1, m, lam, M=M, o=o, Lw=Lw)
        ref = oracle.conv_unequal(f, g, m, lam, M=M, o=o, Lw=Lw)
        assert rel_max_err(h, ref) < TOL64, (m, lam, M, o, Lw)


def test_equal_lengths_lam1_match_convnd_bitwise(hdc):
    L = 1000
    f = synth.unit_disk(21, (3, L))
    g = synth.unit_disk(22, (3, L))
    for m, D in ((512, 1), (1024, 0), (250, 3)):
        a = run(hdc, f, g, 1, m, 1, D=D)
        b = hdc.convnd(dev(f), dev(g), 1, m, D=D).cpu().numpy()
        assert np.array_equal(a, b), (m, D)


def test_fused_and_split_routes(hdc):
    """lam m at and above the single-tile limit (2048 points in FP64) and
    far below it: both routes, against O2 on the padded inputs."""
    cases = [(3000, 20000, 1024, 4), (3000, 20000, 512, 2), (700, 9000, 128, 16), (4096, 16384, 2048, 2),
             (100, 50000, 64, 64), (20000, 3000, 1024, 2)]
    for Lf, Lg, m, lam in cases:
        f = synth.unit_disk(300 + Lf, (Lf,))
        g = synth.unit_disk(400 + Lg, (Lg,))
        h = run(hdc, f, g, 1, m, lam)
        ref = full_conv(f, g, 1, "fft")[:Lg]
        assert rel_max_err(h, ref) < TOL64, (Lf, Lg, m, lam)


def test_passes_and_batch(hdc):
    f = synth.unit_disk(41, (5, 300))
    g = synth.unit_disk(42, (5, 2500))
    ref = full_conv(f, g, 1, "fft")[:, :2500]
    for m, lam, D in ((64, 4, 1), (64, 4, 3), (100, 3, 2), (512, 8, 1)):
        h = run(hdc, f, g, 1, m, lam, D=D)
        assert rel_max_err(h, ref) < TOL64, (m, lam, D)


def test_exact_integers(hdc):
    Lf, Lg = 300, 5000
    fre, fim = synth.small_ints(51, (Lf,))
    gre, gim = synth.small_ints(52, (Lg,))
    pad_re = np.zeros(Lg, dtype=np.int64)
    pad_im = np.zeros(Lg, dtype=np.int64)
    pad_re[:Lf], pad_im[:Lf] = fre, fim
    hre, him = oracle.conv_int_exact(pad_re, pad_im, gre, gim)
    for m, lam in ((64, 8), (300, 1), (128, 16)):
        h = run(hdc, fre + 1j * fim, gre + 1j * gim, 1, m, lam)
        assert np.array_equal(np.rint(h.real).astype(np.int64), hre), (m, lam)
        assert np.array_equal(np.rint(h.imag).astype(np.int64), him), (m, lam)


def test_single_tap_and_fp32(hdc):
    g = synth.unit_disk(61, (777,))
    f = synth.unit_disk(62, (1,))
    h = run(hdc, f, g, 1, 1, 4)
    assert rel_max_err(h, f[0] * g) < TOL64
    f = synth.unit_disk(63, (3, 200))
    g = synth.unit_disk(64, (3, 3000))
    ref = full_conv(f, g, 1, "fft")[:, :3000]
    for m, lam in ((64, 4), (256, 16), (1024, 8)):
        h = run(hdc, f, g, 1, m, lam, dtype=np.complex64)
        assert rel_max_err(h, ref) < TOL32, (m, lam)


def test_full_size_sampled(hdc):
    """Lg = 2^22 with Lf = 2^12 (m = 4096, lam = 512: the split route with
    two-point column transforms for f), sampled outputs against O1."""
    Lf, Lg = 1 << 12, 1 << 22
    f = synth.unit_disk(71, (Lf,))
    g = synth.unit_disk(72, (Lg,))
    h = run(hdc, f, g, 1, 4096, 512)
    fp = np.zeros(Lg, dtype=complex)
    fp[:Lf] = f
    rng = np.random.default_rng(7)
    idx = np.concatenate([[0, 1, Lf - 1, Lf, Lg - 1], rng.integers(0, Lg, 59)]).astype(np.int64)
    ref = oracle.conv_direct_at(fp, g, idx)
    assert rel_max_err(h[idx], ref) < TOL64


# ----------------------------------------------------------------- N-D

def test_2d_against_direct(hdc):
    f = synth.unit_disk(81, (2, 9, 12))
    g = synth.unit_disk(82, (2, 30, 40))
    full = full_conv(f, g, 2)
    for m, lam, D in (((8, 4), (2, 5), (0, 0)), ((4, 4), (4, 2), (1, 2)), ((16, 16), (1, 1), (0, 0)),
                      ((3, 5), (3, 7), (2, 0))):
        h = run(hdc, f, g, 2, list(m), list(lam), D=list(D))
        assert rel_max_err(h, full[:, :30, :40]) < TOL64, (m, lam, D)


def test_2d_window_and_fp32(hdc):
    f = synth.unit_disk(83, (20, 6))
    g = synth.unit_disk(84, (50, 64))
    full = full_conv(f, g, 2)
    h = run(hdc, f, g, 2, [16, 4], [4, 4], o=[5, 3], Lw=[60, 66], M=[80, 80])
    assert rel_max_err(h, full[5:65, 3:69]) < TOL64
    h = run(hdc, f, g, 2, [16, 4], [4, 4], dtype=np.complex64)
    assert rel_max_err(h, full[:50, :64]) < TOL32


def test_3d_against_direct(hdc):
    f = synth.unit_disk(91, (3, 4, 5))
    g = synth.unit_disk(92, (6, 7, 8))
    full = full_conv(f, g, 3)
    for m, lam in (((2, 4, 3), (2, 1, 3)), ((4, 4, 4), (2, 2, 2)), ((8, 7, 8), (1, 1, 1))):
        h = run(hdc, f, g, 3, list(m), list(lam))
        assert rel_max_err(h, full[:6, :7, :8]) < TOL64, (m, lam)


def test_2d_large_split_inner(hdc):
    """Inner axis on the split route (lam m = 4096 > 2048)."""
    f = synth.unit_disk(93, (5, 600))
    g = synth.unit_disk(94, (12, 7000))
    full = full_conv(f, g, 2, "fft")
    h = run(hdc, f, g, 2, [8, 512], [2, 8])
    assert rel_max_err(h, full[:12, :7000]) < TOL64


# -------------------------------------------------------------- errors

def test_errors(hdc):
    f = dev(synth.unit_disk(1, (7,)))
    g = dev(synth.unit_disk(2, (20,)))
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_unequal(f, g, 1, 4, 2, M=25)
    assert e.value.code == hdc.HDC_ERR_ALIAS
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_unequal(f, g, 1, 4, 11)
    assert e.value.code == hdc.HDC_ERR_UNSUPPORTED_SIZE
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_unequal(f, g, 1, 4, 2, out=g)
    assert e.value.code == hdc.HDC_ERR_PARAM
    with pytest.raises(hdc.HDCError) as e:
        hdc.convnd_unequal(f, g, 1, 4, 2, o=5, Lw=22, M=40)
    assert e.value.code == hdc.HDC_ERR_PARAM


# --------------------------------------------------------------- tuner

def test_tuner_picks_a_valid_fast_tuple_and_caches(hdc, tmp_path):
    Lf, Lg = 300, 20000
    f = dev(synth.unit_disk(95, (Lf,)))
    g = dev(synth.unit_disk(96, (Lg,)))
    db = str(tmp_path / "tune.txt")
    best, trials = hdc.tune_unequal(f, g, 1, reps=2, tuning_db=db)
    assert trials and all(t[0]["ms"] > 0 for t in trials)
    b = best[0]
    check_best_timed(best, trials)
    h = hdc.convnd_unequal(f, g, 1, b["m"], b["lam"], D=b["D"]).cpu().numpy()
    ref = full_conv(f.cpu().numpy(), g.cpu().numpy(), 1, "fft")[:Lg]
    assert rel_max_err(h, ref) < TOL64
    again, tr2 = hdc.tune_unequal(f, g, 1, reps=2, tuning_db=db)
    assert tr2 == [] and (again[0]["m"], again[0]["lam"], again[0]["D"]) == (b["m"], b["lam"], b["D"])

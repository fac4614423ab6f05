"""Pins for the CPU oracle: each oracle routine is checked against something
other than itself -- a library routine, a closed form, a brute-force sum in
high precision, an exact integer result, or a value printed in the paper.

Runs on CPU (not marked gpu).
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.signal

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- roots

def test_root_of_unity_matches_numpy_exp():
    rng = np.random.default_rng(0)
    for n in [1, 2, 3, 5, 7, 8, 12, 1000, 2047, 4096, 3 * 2 ** 20, 2 ** 23]:
        ks = np.unique(np.concatenate([np.arange(min(n, 64)), rng.integers(0, n, 64), [n - 1, n // 2, n // 4, n // 8]]))
        for k in ks:
            z = oracle.root_of_unity(int(k), n)
            ref = np.exp(2j * np.pi * (int(k) / n))
            assert abs(z - ref) < 4e-16 * max(1.0, 2 * np.pi * k / n), (k, n)


def test_orthogonality_golden():
    """Section 2.1 orthogonality, sum_j zeta_M^{l j}, from the golden file."""
    with open(os.path.join(GOLD, "orthogonality.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        M, l = c["M"], c["l"]
        s = sum(oracle.root_of_unity(l * j, M) for j in range(M))
        assert abs(s - c["sum"]) < 1e-12 * M


def test_dft_matches_numpy():
    x = synth.unit_disk(11, (30,))
    # numpy: fft uses exp(-2 pi i kj/n); ifft uses +, scaled 1/n
    assert rel_max_err(oracle.dft(x, +1), np.fft.ifft(x) * x.size) < 1e-14
    assert rel_max_err(oracle.dft(x, -1), np.fft.fft(x)) < 1e-14


# ------------------------------------------------------------- O1 direct

@pytest.mark.parametrize("L", [1, 2, 3, 7, 17, 64, 100, 257])
def test_direct_1d_matches_numpy_convolve(L):
    f = synth.unit_disk(100 + L, (L,))
    g = synth.unit_disk(200 + L, (L,))
    ref = np.convolve(f, g)[:L]
    assert rel_max_err(oracle.conv_direct(f, g), ref) < 1e-15


def test_direct_1d_asymmetric_catches_transposition():
    # f*g = g*f in exact arithmetic, but a reversed index (f_j g_j) or a
    # dropped imaginary cross term would break the numpy pin below.
    f = np.array([1 + 2j, 3 - 1j, 0.5j, -2.0])
    g = np.array([2.0, -1j, 4 + 0.5j, 1 - 1j])
    h = oracle.conv_direct(f, g)
    ref = np.array([f[0] * g[0],
                    f[0] * g[1] + f[1] * g[0],
                    f[0] * g[2] + f[1] * g[1] + f[2] * g[0],
                    f[0] * g[3] + f[1] * g[2] + f[2] * g[1] + f[3] * g[0]])
    assert np.array_equal(h, ref)


@pytest.mark.parametrize("shape", [(5, 7), (16, 16), (1, 9), (9, 1)])
def test_direct_2d_matches_scipy(shape):
    f = synth.unit_disk(5, shape)
    g = synth.unit_disk(6, shape)
    ref = scipy.signal.convolve(f, g, method="direct")[: shape[0], : shape[1]]
    assert rel_max_err(oracle.conv_direct(f, g), ref) < 1e-14


@pytest.mark.parametrize("shape", [(3, 4, 5), (8, 8, 8)])
def test_direct_3d_matches_scipy(shape):
    f = synth.unit_disk(7, shape)
    g = synth.unit_disk(8, shape)
    ref = scipy.signal.convolve(f, g, method="direct")[: shape[0], : shape[1], : shape[2]]
    assert rel_max_err(oracle.conv_direct(f, g), ref) < 1e-14


def test_direct_at_matches_full():
    f = synth.unit_disk(9, (12, 10))
    g = synth.unit_disk(10, (12, 10))
    full = oracle.conv_direct(f, g).ravel()
    idx = np.array([0, 1, 9, 10, 57, 119])
    assert np.array_equal(oracle.conv_direct_at(f, g, idx), full[idx])


def test_direct_high_precision_brute_force():
    """Double-double accumulation agrees with an exact rational sum."""
    from fractions import Fraction
    L = 40
    f = synth.unit_disk(12, (L,))
    g = synth.unit_disk(13, (L,))
    h = oracle.conv_direct(f, g)
    for k in [0, 1, 19, 39]:
        re = sum(Fraction(f[j].real) * Fraction(g[k - j].real) - Fraction(f[j].imag) * Fraction(g[k - j].imag)
                 for j in range(k + 1))
        im = sum(Fraction(f[j].real) * Fraction(g[k - j].imag) + Fraction(f[j].imag) * Fraction(g[k - j].real)
                 for j in range(k + 1))
        assert h[k].real == float(re) and h[k].imag == float(im)


# --------------------------------------------------------- O4 closed forms

def _closed_form_mp(A, B, P, k):
    """sum_{j<=k} zeta_P^{A j} zeta_P^{B (k-j)} summed term by term in 50 digits."""
    import mpmath as mp
    mp.mp.dps = 50
    s = mp.mpc(0)
    for j in range(k + 1):
        e = (A * j + B * (k - j)) % P
        s += mp.expjpi(mp.mpf(2 * e) / P)
    return complex(s)


@pytest.mark.parametrize("A,B,P", [(3, 11, 97), (5, 5, 64), (1, 1000, 4099), (7, 2, 12)])
def test_closed_form_exp_vs_mpmath_sum(A, B, P):
    pytest.importorskip("mpmath")
    L = 150
    h = oracle.closed_form_exp(A, B, P, L)
    for k in [0, 1, 2, 33, 149]:
        ref = _closed_form_mp(A, B, P, k)
        assert abs(h[k] - ref) < 1e-13 * max(1.0, abs(ref))


@pytest.mark.parametrize("L", [1, 5, 200, 1000])
def test_closed_form_exp_pins_direct(L):
    A, B, P = 17, 1234, 10007
    f = synth.exp_seq(A, P, L)
    g = synth.exp_seq(B, P, L)
    cf = oracle.closed_form_exp(A, B, P, L)
    assert rel_max_err(oracle.conv_direct(f, g), cf) < 1e-13


def test_closed_form_equal_frequencies():
    # A = B: h_k = (k+1) zeta^{Bk}
    L = 64
    f = synth.exp_seq(9, 31, L)
    h = oracle.conv_direct(f, f)
    cf = oracle.closed_form_exp(9, 9, 31, L)
    assert rel_max_err(h, cf) < 1e-14
    assert abs(cf[10] - 11 * np.exp(2j * np.pi * (90 % 31) / 31)) < 1e-13


def test_closed_form_geom_pins_direct():
    L = 300
    f = synth.geom_seq(0.97, 3, 101, L)
    g = synth.geom_seq(0.9, 40, 101, L)
    cf = oracle.closed_form_geom(0.97, 3, 0.9, 40, 101, L)
    assert rel_max_err(oracle.conv_direct(f, g), cf) < 1e-13


# ------------------------------------------------------- O2 explicit FFT

@pytest.mark.parametrize("L", [1, 2, 3, 31, 64, 1000, 2048])
def test_fft_conv_1d_vs_direct(L):
    f = synth.unit_disk(300 + L, (L,))
    g = synth.unit_disk(400 + L, (L,))
    assert rel_max_err(oracle.conv_fft(f, g), oracle.conv_direct(f, g)) < 1e-13


@pytest.mark.parametrize("L", [2 ** 16, 3 * 2 ** 14])
def test_fft_conv_1d_vs_closed_form_large(L):
    A, B, P = 12345, 777, 2 ** 20 + 7
    f = synth.exp_seq(A, P, L)
    g = synth.exp_seq(B, P, L)
    assert rel_max_err(oracle.conv_fft(f, g), oracle.closed_form_exp(A, B, P, L)) < 1e-12


@pytest.mark.parametrize("shape", [(6, 9), (33, 17), (5, 6, 7)])
def test_fft_conv_nd_vs_direct_and_numpy(shape):
    f = synth.unit_disk(21, shape)
    g = synth.unit_disk(22, shape)
    h = oracle.conv_fft(f, g)
    assert rel_max_err(h, oracle.conv_direct(f, g)) < 1e-13
    full = [2 * n - 1 for n in shape]
    ax = list(range(len(shape)))
    ref = np.fft.ifftn(np.fft.fftn(f, full, axes=ax) * np.fft.fftn(g, full, axes=ax), axes=ax)[tuple(slice(0, n) for n in shape)]
    assert rel_max_err(h, ref) < 1e-13


def test_fft_conv_2d_separable_closed_form():
    # f(x,y) = a_x b_y separable => h = (a*a')(x) (b*b')(y)
    Lx, Ly, P = 40, 24, 211
    ax, bx = synth.exp_seq(3, P, Lx), synth.exp_seq(50, P, Lx)
    ay, by = synth.exp_seq(7, P, Ly), synth.exp_seq(100, P, Ly)
    f = np.outer(ax, ay)
    g = np.outer(bx, by)
    ref = np.outer(oracle.closed_form_exp(3, 50, P, Lx), oracle.closed_form_exp(7, 100, P, Ly))
    assert rel_max_err(oracle.conv_fft(f, g), ref) < 1e-13
    assert rel_max_err(oracle.conv_direct(f, g), ref) < 1e-13


# ---------------------------------------------------- O3 exact integers

def test_int_exact_direct_vs_numpy():
    L = 500
    fr, fi = synth.small_ints(31, (L,))
    gr, gi = synth.small_ints(32, (L,))
    hr, hi = oracle.conv_int_exact(fr, fi, gr, gi, "direct")
    ref_r = np.convolve(fr, gr)[:L] - np.convolve(fi, gi)[:L]
    ref_i = np.convolve(fr, gi)[:L] + np.convolve(fi, gr)[:L]
    assert np.array_equal(hr, ref_r) and np.array_equal(hi, ref_i)


@pytest.mark.parametrize("L", [1, 2, 1000, 3000])
def test_int_exact_ntt_vs_direct(L):
    fr, fi = synth.small_ints(33 + L, (L,))
    gr, gi = synth.small_ints(34 + L, (L,))
    a = oracle.conv_int_exact(fr, fi, gr, gi, "direct")
    b = oracle.conv_int_exact(fr, fi, gr, gi, "ntt")
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_int_exact_ntt_extreme_values():
    # all +8 / -8: the largest magnitudes the workload allows
    L = 2 ** 15
    fr = np.full(L, 8)
    fi = np.full(L, -8)
    gr = np.full(L, -8)
    gi = np.full(L, 8)
    hr, hi = oracle.conv_int_exact(fr, fi, gr, gi, "ntt")
    k = np.arange(L)
    # (8-8i)(-8+8i) = -64+64i+64i+64 = 128i per term
    assert np.array_equal(hr, np.zeros(L, dtype=np.int64))
    assert np.array_equal(hi, 128 * (k + 1))


def test_int_exact_matches_fft_rounded():
    L = 2 ** 14
    fr, fi = synth.small_ints(40, (L,))
    gr, gi = synth.small_ints(41, (L,))
    hr, hi = oracle.conv_int_exact(fr, fi, gr, gi, "ntt")
    h = oracle.conv_fft(synth.ints_to_complex(fr, fi), synth.ints_to_complex(gr, gi))
    assert np.array_equal(np.rint(h.real).astype(np.int64), hr)
    assert np.array_equal(np.rint(h.imag).astype(np.int64), hi)


# ------------------------------------------- O5 residue transforms (Eq. 1, 2)

def _padded_dft_plus(x, N):
    """sum_j zeta_N^{+kj} x_j of x zero-padded to N (numpy library route)."""
    return np.fft.ifft(x, N) * N


@pytest.mark.parametrize("L,m,p,q", [(6, 4, 2, 3), (5, 5, 1, 2), (8, 2, 4, 8), (7, 3, 3, 5), (12, 12, 1, 1),
                                      (1, 1, 1, 1), (10, 4, 3, 6)])
def test_residue_forward_is_padded_dft(L, m, p, q):
    x = synth.unit_disk(50 + L, (L,))
    F = oracle.residue_forward(x, L, m, p, q)
    assert rel_max_err(F, _padded_dft_plus(x, q * m)) < 1e-13


@pytest.mark.parametrize("L,m,p,q", [(6, 4, 2, 3), (7, 3, 3, 5), (10, 4, 3, 6), (9, 9, 1, 2)])
def test_residue_backward_round_trip(L, m, p, q):
    x = synth.unit_disk(60 + L, (L,))
    F = oracle.residue_forward(x, L, m, p, q)
    y = oracle.residue_backward(F, L, m, p, q)
    assert rel_max_err(y, x) < 1e-13
    # and Eq. 2 against the library inverse DFT of an arbitrary spectrum
    N = q * m
    G = synth.unit_disk(70 + L, (N,))
    assert rel_max_err(oracle.residue_backward(G, L, m, p, q), np.fft.fft(G)[:L] / N) < 1e-13


def test_hybrid_paper_example():
    """The 1-D parameter example of Section 2.5 (L=6, M=11, m=4, p=2, q=3)."""
    with open(os.path.join(GOLD, "paper_1d_parameter_example.json")) as fh:
        ex = json.load(fh)
    L, m, p, q = ex["L"], ex["m"], ex["p"], ex["q"]
    f = synth.unit_disk(1, (L,))
    g = synth.unit_disk(2, (L,))
    assert q * m >= 2 * L - 1
    assert rel_max_err(oracle.conv_hybrid(f, g, m, p, q), np.convolve(f, g)[:L]) < 1e-14


def _valid_tuples(L, M):
    for m in range(1, M + 1):
        p = -(-L // m)
        q = -(-M // m)
        yield m, p, q


def test_hybrid_brute_force_all_small():
    """Every valid (m, p, q) for every L <= 10 and M in [2L-1, 2L+2] gives
    the direct convolution (Section 3: the decomposition is exact)."""
    for L in range(1, 11):
        f = synth.unit_disk(80 + L, (L,))
        g = synth.unit_disk(90 + L, (L,))
        ref = np.convolve(f, g)[:L]
        for M in range(2 * L - 1, 2 * L + 3):
            for m, p, q in _valid_tuples(L, M):
                h = oracle.conv_hybrid(f, g, m, p, q)
                assert rel_max_err(h, ref) < 1e-13, (L, M, m, p, q)


def test_hybrid_aliasing_when_padding_too_small():
    """With q m < 2L - 1 the result is contaminated by aliases (Section 3.1)."""
    L = 8
    f = synth.unit_disk(3, (L,))
    g = synth.unit_disk(4, (L,))
    ref = np.convolve(f, g)[:L]
    h = oracle.conv_hybrid(f, g, 4, 2, 2)      # q m = 8 < 15
    assert rel_max_err(h, ref) > 1e-3


# ------------------------------------------- O6 centered Hermitian convolution

def _herm_full(a):
    """Full centered (2K-1)^2 spectrum from the stored half (numpy)."""
    K = a.shape[1]
    full = np.zeros((2 * K - 1, 2 * K - 1), dtype=np.complex128)
    c = K - 1
    full[:, c:] = a
    for kx in range(-c, c + 1):
        for ky in range(1, K):
            full[kx + c, c - ky] = np.conj(a[-kx + c, ky])
    return full


@pytest.mark.parametrize("K", [1, 2, 4, 7])
def test_hermitian_direct_vs_scipy_full(K):
    f = synth.hermitian_normal(5, K)
    g = synth.hermitian_normal(6, K)
    F, G = _herm_full(f), _herm_full(g)
    full = scipy.signal.convolve(F, G, method="direct")    # indices shifted by 2c
    c = K - 1
    ref = full[c:c + 2 * K - 1, 2 * c:2 * c + K]
    assert rel_max_err(oracle.conv_hermitian_direct(f, g), ref) < 1e-13


@pytest.mark.parametrize("K", [3, 8, 16])
def test_hermitian_fft_vs_direct(K):
    f = synth.hermitian_normal(7, K)
    g = synth.hermitian_normal(8, K)
    h = oracle.conv_hermitian_fft(f, g)
    assert rel_max_err(h, oracle.conv_hermitian_direct(f, g)) < 1e-13
    # the product of real fields is real: its half-spectrum is Hermitian on ky=0
    c = K - 1
    assert np.allclose(h[::-1, 0], np.conj(h[:, 0]), atol=1e-12)
    assert abs(h[c, 0].imag) < 1e-12

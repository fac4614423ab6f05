"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: relative max-norm error <= 1e-12 in FP64 and <= 5e-5 in FP32
against the FP64 oracle; integer-valued FP64 inputs must round to the exact
integer convolution bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err

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


def run(hdc, f, g, dims, m, p=0, q=0, D=0, M=None, dtype=np.complex128, **kw):
    tdt = torch.complex128 if dtype == np.complex128 else torch.complex64
    ft = torch.from_numpy(np.ascontiguousarray(f, dtype=dtype)).to("cuda", tdt)
    gt = torch.from_numpy(np.ascontiguousarray(g, dtype=dtype)).to("cuda", tdt)
    h = hdc.convnd(ft, gt, dims, m, M=M, p=p, q=q, D=D, **kw)
    torch.cuda.synchronize()
    return h.cpu().numpy().astype(np.complex128)


def good_sizes(lo, hi):
    out = []
    for n in range(lo, hi + 1):
        k = n
        for f in (2, 3, 5, 7):
            while k % f == 0:
                k //= f
        if k == 1:
            out.append(n)
    return out


# ------------------------------------------------------------------ 1-D

def test_brute_force_all_tuples_tiny(hdc):
    """Every valid (m, p, q) with D in {1, q} for L <= 12, M in {2L-1, 2L}."""
    for L in range(1, 13):
        f = synth.unit_disk(1000 + L, (L,))
        g = synth.unit_disk(2000 + L, (L,))
        ref = oracle.conv_direct(f, g)
        for M in (2 * L - 1, 2 * L):
            for m in good_sizes(1, hdc.next_good_size(M)):
                q = -(-M // m)
                for D in sorted({1, q}):
                    h = run(hdc, f, g, 1, m, M=M, D=D)
                    assert rel_max_err(h, ref) < TOL64, (L, M, m, D)


def test_paper_parameter_example(hdc):
    L, M, m = 6, 11, 4            # Section 2.5 figure: p = 2, q = 3
    f = synth.unit_disk(6, (L,))
    g = synth.unit_disk(7, (L,))
    h = run(hdc, f, g, 1, m, M=M, p=2, q=3)
    assert rel_max_err(h, oracle.conv_direct(f, g)) < TOL64


def test_config1_L1024_m512(hdc):
    """L=1024, M=2047, m=512, D=1 (p=2, q=4 derived); the literal p=1 is rejected."""
    L = 1024
    f = synth.unit_disk(synth.BASE_SEED + 1, (L,))
    g = synth.unit_disk(synth.BASE_SEED + 101, (L,))
    ref = oracle.conv_direct(f, g)
    h = run(hdc, f, g, 1, 512, M=2047, D=1)
    assert rel_max_err(h, ref) < TOL64
    with pytest.raises(hdc.HDCError) as ei:
        run(hdc, f, g, 1, 512, M=2047, p=1, q=4, D=1)
    assert ei.value.code == hdc.HDC_ERR_PARAM
    # the nearest valid p = 1 tuple
    h = run(hdc, f, g, 1, 1024, M=2047, p=1, q=2, D=1)
    assert rel_max_err(h, ref) < TOL64


RAGGED = [
    # (L, m, D): ragged tails (L not a multiple of m), several passes (D < q)
    (1000, 256, 1), (1000, 250, 3), (1000, 2000, 1), (3001, 1024, 2), (3001, 768, 0),
    (4097, 4096, 1), (4097, 2187, 0), (5000, 3000, 2), (777, 49, 5), (2048, 4096, 0),
]


@pytest.mark.parametrize("L,m,D", RAGGED)
def test_ragged_fp64(hdc, L, m, D):
    f = synth.unit_disk(3000 + L, (L,))
    g = synth.unit_disk(4000 + L, (L,))
    ref = oracle.conv_direct(f, g)
    assert rel_max_err(run(hdc, f, g, 1, m, D=D), ref) < TOL64


@pytest.mark.parametrize("L,m,D", RAGGED)
def test_ragged_fp32(hdc, L, m, D):
    f = synth.unit_disk(3000 + L, (L,))
    g = synth.unit_disk(4000 + L, (L,))
    ref = oracle.conv_direct(f, g)
    assert rel_max_err(run(hdc, f, g, 1, m, D=D, dtype=np.complex64), ref) < TOL32


# m beyond one shared-memory tile: the split m = m1 m2 route
SPLIT = [(20000, 1 << 15, 0), (20000, 12288, 1), (9000, 5000, 0), (70000, 1 << 17, 1), (65536, 65536, 0)]


@pytest.mark.parametrize("L,m,D", SPLIT)
def test_split_route_fp64(hdc, L, m, D):
    f = synth.unit_disk(5000 + L, (L,))
    g = synth.unit_disk(6000 + L, (L,))
    ref = oracle.conv_fft(f, g)
    h = run(hdc, f, g, 1, m, D=D)
    assert rel_max_err(h, ref) < TOL64
    idx = np.array([0, 1, L // 3, L - 2, L - 1])
    assert rel_max_err(h[idx], oracle.conv_direct_at(f, g, idx)) < TOL64


@pytest.mark.parametrize("L,m,D", SPLIT[:3])
def test_split_route_fp32(hdc, L, m, D):
    f = synth.unit_disk(5000 + L, (L,))
    g = synth.unit_disk(6000 + L, (L,))
    assert rel_max_err(run(hdc, f, g, 1, m, D=D, dtype=np.complex64), oracle.conv_fft(f, g)) < TOL32


def test_explicit_and_implicit_special_cases(hdc):
    L = 1536
    M = 2 * L - 1
    f = synth.unit_disk(71, (L,))
    g = synth.unit_disk(72, (L,))
    ref = oracle.conv_direct(f, g)
    m, p, q = hdc.explicit_params(L, M)                 # explicit: q = 1
    assert rel_max_err(run(hdc, f, g, 1, m, p=p, q=q, M=M), ref) < TOL64
    assert rel_max_err(run(hdc, f, g, 1, 768, M=2 * L), ref) < TOL64   # implicit: L=2m, M=4m


def test_every_tuple_same_result(hdc):
    """Invariance: all valid (m, D) at one (L, M) agree with each other."""
    L, M = 3000, 5999
    f = synth.unit_disk(81, (L,))
    g = synth.unit_disk(82, (L,))
    ref = oracle.conv_direct(f, g)
    outs = []
    for m in [6000, 3000, 2048, 1536, 1000, 750, 512, 375, 125, 60, 6144, 8192]:
        q = -(-M // m)
        for D in sorted({1, q}):
            h = run(hdc, f, g, 1, m, M=M, D=D)
            assert rel_max_err(h, ref) < TOL64, (m, D)
            outs.append(h)
    for h in outs[1:]:
        assert rel_max_err(h, outs[0]) < 2 * TOL64


@pytest.mark.parametrize("L,m", [(4096, 1024), (1 << 16, 1 << 15), (3 * (1 << 14), 1 << 14), (50000, 12500)])
def test_integer_inputs_bit_exact(hdc, L, m):
    fr, fi = synth.small_ints(91 + L, (L,))
    gr, gi = synth.small_ints(92 + L, (L,))
    hr, hi = oracle.conv_int_exact(fr, fi, gr, gi)
    h = run(hdc, synth.ints_to_complex(fr, fi), synth.ints_to_complex(gr, gi), 1, m)
    assert np.array_equal(np.rint(h.real).astype(np.int64), hr)
    assert np.array_equal(np.rint(h.imag).astype(np.int64), hi)
    assert np.max(np.abs(h - (hr + 1j * hi))) < 1e-3


def test_batch_rows(hdc):
    B, L = 5, 700
    f = synth.unit_disk(101, (B, L))
    g = synth.unit_disk(102, (B, L))
    h = run(hdc, f, g, 1, 350, D=2)
    for b in range(B):
        assert rel_max_err(h[b], oracle.conv_direct(f[b], g[b])) < TOL64


def test_inplace(hdc):
    L = 1000
    f = synth.unit_disk(111, (L,))
    g = synth.unit_disk(112, (L,))
    ft = torch.from_numpy(f).cuda()
    gt = torch.from_numpy(g).cuda()
    out = hdc.conv1d(ft, gt, 256, D=1, inplace=True)
    torch.cuda.synchronize()
    assert out.data_ptr() == ft.data_ptr()
    assert rel_max_err(ft.cpu().numpy(), oracle.conv_direct(f, g)) < TOL64
    # f * f in place (both inputs alias the output)
    ft = torch.from_numpy(f).cuda()
    hdc.conv1d(ft, ft, 300, D=2, inplace=True)
    torch.cuda.synchronize()
    assert rel_max_err(ft.cpu().numpy(), oracle.conv_direct(f, f)) < TOL64


def test_empty_batch(hdc):
    ft = torch.zeros((0, 64), dtype=torch.complex128, device="cuda")
    h = hdc.conv1d(ft, ft, 64)
    assert h.shape == (0, 64)


# ------------------------------------------------------------- 2-D / 3-D

ND = [
    ((33, 47), (32, 48), 0), ((64, 64), (64, 128), 1), ((64, 64), (128, 32), 0), ((17, 5), (9, 9), 1),
    ((1, 40), (1, 80), 0), ((9, 10, 11), (6, 20, 7), 0), ((16, 16, 16), (32, 16, 8), 1),
]


@pytest.mark.parametrize("shape,m,D", ND)
def test_nd_fp64(hdc, shape, m, D):
    f = synth.unit_disk(121, shape)
    g = synth.unit_disk(122, shape)
    ref = oracle.conv_direct(f, g)
    assert rel_max_err(run(hdc, f, g, len(shape), list(m), D=D), ref) < TOL64


@pytest.mark.parametrize("shape,m,D", ND)
def test_nd_fp32(hdc, shape, m, D):
    f = synth.unit_disk(121, shape)
    g = synth.unit_disk(122, shape)
    ref = oracle.conv_direct(f, g)
    assert rel_max_err(run(hdc, f, g, len(shape), list(m), D=D, dtype=np.complex64), ref) < TOL32


def test_2d_separable_closed_form(hdc):
    Lx, Ly, P = 300, 200, 1009
    f = np.outer(synth.exp_seq(3, P, Lx), synth.exp_seq(7, P, Ly))
    g = np.outer(synth.exp_seq(50, P, Lx), synth.exp_seq(100, P, Ly))
    ref = np.outer(oracle.closed_form_exp(3, 50, P, Lx), oracle.closed_form_exp(7, 100, P, Ly))
    assert rel_max_err(run(hdc, f, g, 2, [150, 256]), ref) < TOL64


# --------------------------------------------- full sizes (sampled checks)

@pytest.mark.parametrize("L,m", [(1 << 20, 1 << 19), (1 << 22, 1 << 21), (3 << 20, 3 << 19), (1 << 22, 1 << 22)])
def test_large_closed_form_fp64(hdc, L, m):
    A, B, P = 123457, 98765, (1 << 26) + 7
    f = synth.exp_seq(A, P, L)
    g = synth.exp_seq(B, P, L)
    h = run(hdc, f, g, 1, m)
    assert rel_max_err(h, oracle.closed_form_exp(A, B, P, L)) < TOL64


def test_large_sampled_unit_disk_fp64(hdc):
    L = 1 << 22
    f = synth.unit_disk(synth.BASE_SEED + 2, (L,))
    g = synth.unit_disk(synth.BASE_SEED + 102, (L,))
    h = run(hdc, f, g, 1, 1 << 21)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, 1, L - 1], rng.integers(0, L, 13)]))
    ref = oracle.conv_direct_at(f, g, idx)
    # relative to the largest sampled value of the reference
    assert np.max(np.abs(h[idx] - ref)) < TOL64 * np.max(np.abs(ref))


def test_large_integer_bit_exact(hdc):
    L = 1 << 22
    fr, fi = synth.small_ints(synth.BASE_SEED + 3, (L,))
    gr, gi = synth.small_ints(synth.BASE_SEED + 103, (L,))
    hr, hi = oracle.conv_int_exact(fr, fi, gr, gi, "ntt")
    h = run(hdc, synth.ints_to_complex(fr, fi), synth.ints_to_complex(gr, gi), 1, 1 << 21)
    assert np.array_equal(np.rint(h.real).astype(np.int64), hr)
    assert np.array_equal(np.rint(h.imag).astype(np.int64), hi)


def test_fused_inverse_unfold_against_separate_passes(hdc):
    """Split-route sizes with enough column tiles (m1 = 320 or 512 columns
    of 2048-point rows) and one residue per pass take the fused inverse +
    unfold kernel; their results match the oracle, beside several residues
    per pass (the separate passes) and a window that starts past the input
    length."""
    hdc.stats_reset()
    hdc.stats_timing(True)
    L = 600000
    f = synth.unit_disk(5101, (L,))
    g = synth.unit_disk(5102, (L,))
    fp = np.concatenate([f, np.zeros(L, dtype=complex)])
    gp = np.concatenate([g, np.zeros(L, dtype=complex)])
    full = oracle.conv_fft(fp, gp)
    for m, D in ((1048576, 0), (1048576, 1), (655360, 0)):
        h = run(hdc, f, g, 1, m, D=D)
        assert rel_max_err(h, full[:L]) < TOL64, (m, D)
    ft = torch.from_numpy(f).cuda()
    gt = torch.from_numpy(g).cuda()
    hw = hdc.convnd_window(ft, gt, 1, 1048576, 200000, 700000, M=2 * L - 1).cpu().numpy()
    assert rel_max_err(hw, full[200000:900000]) < TOL64
    torch.cuda.synchronize()
    hdc.stats_timing(False)
    assert hdc.stats()["k_ifft_unfold_cols"]["launches"] > 0


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
def test_maximum_transform_size(hdc, dtype):
    """The largest transform of each dtype (2^23 points in FP64, 2^25 in
    FP32, one split into the largest row and column tiles): L = m / 2 with
    q = 1 and L = m with q = 2, sampled outputs against O1; one size more is
    rejected."""
    dt = hdc.HDC_C128 if dtype == np.complex128 else hdc.HDC_C64
    mx = hdc.max_fft_size(dt)
    tol = TOL64 if dtype == np.complex128 else TOL32
    rng = np.random.default_rng(11)
    for L, q in ((mx // 2, 1), (mx, 2)):
        f = synth.unit_disk(5201, (L,))
        g = synth.unit_disk(5202, (L,))
        h = run(hdc, f, g, 1, mx, dtype=dtype)
        idx = np.concatenate([[0, 1, L - 1], rng.integers(0, L, 21)]).astype(np.int64)
        assert rel_max_err(h[idx], oracle.conv_direct_at(f, g, idx)) < tol, (L, q)
    assert hdc.validate_axis(mx, 2 * mx - 1, 2 * mx, dtype=dt)[0] == hdc.HDC_ERR_UNSUPPORTED_SIZE


def test_brute_force_all_tuples_up_to_64(hdc):
    """Every L <= 64, M in {2L-1, 2L+1, 3L, 4L}, every valid m up to
    nextgood(M), D in {1, 2, q}: FP64 against O1 within 1e-12, and for
    integer inputs the rounded result equals the exact convolution for every
    tuple (every tuple gives the same integers)."""
    n = 0
    for L in range(1, 65):
        f = synth.unit_disk(7000 + L, (L,))
        g = synth.unit_disk(8000 + L, (L,))
        ref = oracle.conv_direct(f, g)
        fre, fim = synth.small_ints(9000 + L, (L,))
        gre, gim = synth.small_ints(9500 + L, (L,))
        ire, iim = oracle.conv_int_exact(fre, fim, gre, gim, method="direct")
        fi = fre + 1j * fim
        gi = gre + 1j * gim
        for M in sorted({2 * L - 1, 2 * L + 1, 3 * L, 4 * L}):
            for m in good_sizes(1, hdc.next_good_size(M)):
                q = -(-M // m)
                for D in sorted({1, min(2, q), q}):
                    h = run(hdc, f, g, 1, m, M=M, D=D)
                    assert rel_max_err(h, ref) < TOL64, (L, M, m, D)
                    n += 1
                hi = run(hdc, fi, gi, 1, m, M=M)
                assert np.array_equal(np.rint(hi.real).astype(np.int64), ire), (L, M, m)
                assert np.array_equal(np.rint(hi.imag).astype(np.int64), iim), (L, M, m)
    assert n > 20000

"""Pins of the unequal-length oracle (O8, Section 3.5) to facts outside it.

* the residue-matching index identity qg lg + rg = qf lf + rf, checked
  exhaustively as a bijection of (residue, bin) pairs;
* the direct convolution (O1, itself pinned to library routines) and
  numpy's convolution on random inputs, all windows;
* exact integer convolution (O3) for integer inputs;
* the powers-of-two example of Section 3.4 (M = 2 L2 = 2^a L1, A0 / A1
  interleaving), written out here with explicit DFT sums.
"""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err


def test_residue_matching_identity_exhaustive():
    """For every qg, lam, m: (rg, lg) -> (rf = qg (lg mod lam) + rg,
    lf = lg div lam) maps [0, qg) x [0, lam m) one-to-one onto
    [0, lam qg) x [0, m) and keeps the DFT index."""
    for qg in range(1, 7):
        for lam in range(1, 6):
            for m in range(1, 8):
                qf = lam * qg
                seen = set()
                for rg in range(qg):
                    for lg in range(lam * m):
                        lf, l = divmod(lg, lam)
                        rf = qg * l + rg
                        assert 0 <= rf < qf and 0 <= lf < m
                        assert qg * lg + rg == qf * lf + rf
                        seen.add((rf, lf))
                assert len(seen) == qf * m


def _cases():
    # (Lf, Lg, m, lam, M, o, Lw); M None = least alias-free, Lw None = Lg
    return [
        (1, 1, 1, 1, None, 0, None),
        (1, 9, 2, 3, None, 0, None),
        (5, 5, 4, 1, None, 0, None),
        (7, 20, 4, 2, None, 0, None),
        (7, 20, 2, 4, None, 0, None),
        (7, 20, 3, 2, None, 0, None),
        (7, 20, 5, 1, 40, 0, None),
        (13, 31, 4, 3, None, 0, 43),
        (13, 31, 4, 3, 60, 10, 33),
        (20, 7, 6, 1, None, 0, None),   # f longer than g
        (16, 64, 8, 4, 128, 0, 64),     # powers of two
        (3, 50, 1, 7, None, 0, None),
    ]


@pytest.mark.parametrize("case", _cases())
def test_o8_against_direct_and_numpy(case):
    Lf, Lg, m, lam, M, o, Lw = case
    f = synth.unit_disk(31 + Lf, (Lf,))
    g = synth.unit_disk(37 + Lg, (Lg,))
    full = np.convolve(f, g)
    Lw_ = Lg if Lw is None else Lw
    h = oracle.conv_unequal(f, g, m, lam, M=M, o=o, Lw=Lw)
    want = full[o:o + Lw_]
    assert rel_max_err(h, want) < 1e-13
    # O1 on inputs zero-padded to the length of the linear convolution
    S = Lf + Lg - 1
    fp = np.zeros(S, dtype=complex)
    gp = np.zeros(S, dtype=complex)
    fp[:Lf] = f
    gp[:Lg] = g
    direct = oracle.conv_direct(fp, gp)
    assert rel_max_err(h, direct[o:o + Lw_]) < 1e-13


def test_o8_rejects_aliasing_and_bad_windows():
    f = synth.unit_disk(1, (7,))
    g = synth.unit_disk(2, (20,))
    with pytest.raises(RuntimeError):
        oracle.conv_unequal(f, g, 4, 2, M=25)          # M < Lf + Lg - 1
    with pytest.raises(RuntimeError):
        oracle.conv_unequal(f, g, 4, 2, M=26, o=5, Lw=22)   # past the end
    with pytest.raises(RuntimeError):
        oracle.conv_unequal(f, g, 4, 2, o=5, Lw=21)    # o + Lw > N = 24


def test_o8_exact_integers():
    Lf, Lg = 57, 300
    fre, fim = synth.small_ints(5, (Lf,))
    gre, gim = synth.small_ints(7, (Lg,))
    f = fre + 1j * fim
    g = gre + 1j * gim
    pad = np.zeros(Lg, dtype=np.int64)
    fre_p, fim_p = pad.copy(), pad.copy()
    fre_p[:Lf], fim_p[:Lf] = fre, fim
    hre, him = oracle.conv_int_exact(fre_p, fim_p, gre, gim, method="direct")
    for m, lam in ((16, 4), (20, 3), (64, 1), (7, 7)):
        h = oracle.conv_unequal(f, g, m, lam)
        assert np.array_equal(np.rint(h.real).astype(np.int64), hre)
        assert np.array_equal(np.rint(h.imag).astype(np.int64), him)
        assert np.max(np.abs(h - (hre + 1j * him))) < 1e-9


def _zeta(n, k):
    return np.exp(2j * np.pi * np.asarray(k, dtype=float) / n)


@pytest.mark.parametrize("alpha,L1", [(1, 4), (2, 4), (3, 4), (3, 5)])
def test_powers_of_two_example(alpha, L1):
    """Section 3.4: M = 2 L2 = 2^alpha L1.  f splits into 2^alpha residue
    transforms of L1 points, g into 2 of L2 points; A0 interleaves the even
    residues of f, A1 the odd ones; H0 = A0 G0, H1 = A1 G1; then
    M h_k = sum_j zeta_L2^{-kj} H0_j + zeta_M^{-k} sum_j zeta_L2^{-kj} H1_j,
    k < L2.  That is the oracle's O8 with m = L1, lam = L2 / L1 = 2^(alpha-1)."""
    L2 = (2 ** alpha) * L1 // 2
    M = 2 * L2
    f = synth.unit_disk(400 + alpha, (L1,))
    g = synth.unit_disk(500 + alpha, (L2,))
    j1 = np.arange(L1)
    j2 = np.arange(L2)
    Fres = [np.array([np.sum(_zeta(L1, k * j1) * _zeta(M, i * j1) * f) for k in range(L1)])
            for i in range(2 ** alpha)]
    G0 = np.array([np.sum(_zeta(L2, k * j2) * g) for k in range(L2)])
    G1 = np.array([np.sum(_zeta(L2, k * j2) * _zeta(M, j2) * g) for k in range(L2)])
    lam = 2 ** (alpha - 1)
    A0 = np.empty(L2, dtype=complex)
    A1 = np.empty(L2, dtype=complex)
    for k in range(L1):
        for l in range(lam):
            A0[lam * k + l] = Fres[2 * l][k]
            A1[lam * k + l] = Fres[2 * l + 1][k]
    H0 = A0 * G0
    H1 = A1 * G1
    h = np.array([(np.sum(_zeta(L2, -k * j2) * H0) + _zeta(M, -k) * np.sum(_zeta(L2, -k * j2) * H1)) / M
                  for k in range(L2)])
    want = np.convolve(f, g)[:L2]
    assert rel_max_err(h, want) < 1e-13
    o8 = oracle.conv_unequal(f, g, L1, lam, M=M)
    assert rel_max_err(o8, h) < 1e-13

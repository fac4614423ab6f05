"""Pins of the real-input oracle (O10): convolution of real sequences
through the packed sequence z = f + i g and conjugate residue pairs.

* numpy's convolution (library) and O1 on real inputs;
* every valid (m, p, q) for L <= 10 (even and odd q, self-paired residues
  r = 0 and r = q / 2);
* exact integer convolution (O3) for integer inputs;
* the closed form (k + 1) a^k for two copies of a^j;
* the two-input hybrid O5 on the same inputs as complex arrays.
"""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err


def real_inputs(seed, L):
    z = synth.unit_disk(seed, (L,))
    return z.real.copy(), z.imag.copy()


@pytest.mark.parametrize("L,m", [(1, 1), (2, 3), (7, 4), (7, 13), (16, 8), (31, 7), (64, 127), (100, 50),
                                 (128, 64), (129, 256)])
def test_o10_against_numpy_and_direct(L, m):
    f, g = real_inputs(500 + L, L)
    h = oracle.conv_real(f, g, m)
    assert rel_max_err(h, np.convolve(f, g)[:L]) < 1e-13
    assert rel_max_err(h, oracle.conv_direct(f.astype(complex), g.astype(complex)).real) < 1e-13


def test_o10_every_valid_tuple_tiny():
    for L in range(1, 11):
        f, g = real_inputs(600 + L, L)
        want = np.convolve(f, g)[:L]
        M = 2 * L - 1
        for m in range(1, 2 * M + 1):
            p0, q0 = -(-L // m), -(-M // m)
            for p, q in ((p0, q0), (p0 + 1, q0 + 1)):
                assert rel_max_err(oracle.conv_real(f, g, m, p, q), want) < 1e-13, (L, m, p, q)


def test_o10_exact_integers():
    L = 500
    fre, _ = synth.small_ints(701, (L,))
    gre, _ = synth.small_ints(702, (L,))
    zero = np.zeros(L, dtype=np.int64)
    hre, _ = oracle.conv_int_exact(fre, zero, gre, zero)
    for m in (64, 999, 250):
        h = oracle.conv_real(fre.astype(float), gre.astype(float), m)
        assert np.array_equal(np.rint(h).astype(np.int64), hre), m


def test_o10_closed_form_and_o5():
    L = 80
    a = 0.93
    x = a ** np.arange(L)
    want = (np.arange(L) + 1) * a ** np.arange(L)
    for m in (16, 40, 159, 81):
        assert rel_max_err(oracle.conv_real(x, x, m), want) < 1e-13, m
    f, g = real_inputs(703, 40)
    for m, p, q in ((8, 5, 10), (16, 3, 5), (79, 1, 1)):
        hc = oracle.conv_hybrid(f.astype(complex), g.astype(complex), m, p, q)
        assert np.max(np.abs(hc.imag)) < 1e-13
        assert rel_max_err(oracle.conv_real(f, g, m, p, q), hc.real) < 1e-13


def test_o10_rejects_aliasing():
    f, g = real_inputs(704, 10)
    with pytest.raises(RuntimeError):
        oracle.conv_real(f, g, 6, 2, 3)     # q m = 18 < 2 L - 1

"""Pins of the multi-convolution oracle (O9): the n-fold convolution of n
arrays and the sum of pairwise convolutions, first L outputs.

* iterated numpy convolution (library) and iterated O1 (direct sums);
* exact integer n-fold convolution (iterated O3);
* closed form: n copies of a^j give binom(k + n - 1, n - 1) a^k;
* n = 2 equals O5's two-input hybrid convolution; n = 1 is the identity;
* aliasing: q m below n (L - 1) + 1 is rejected (2 L - 1, enough for two
  inputs, is not enough for three).
"""
from functools import reduce
from math import comb

import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err


def first_L_iterated(xs):
    L = xs.shape[1]
    return reduce(lambda a, b: np.convolve(a, b)[:L], list(xs))


@pytest.mark.parametrize("n,L,m", [(3, 10, 4), (3, 10, 28), (4, 7, 5), (5, 12, 8), (6, 3, 2), (2, 9, 6),
                                   (3, 33, 16), (8, 5, 7)])
def test_o9_against_iterated_library_and_direct(n, L, m):
    xs = synth.unit_disk(700 + 10 * n + L, (n, L))
    h = oracle.conv_multi(xs, m)
    assert rel_max_err(h, first_L_iterated(xs)) < 1e-13
    direct = reduce(lambda a, b: oracle.conv_direct(a, b), list(xs))
    assert rel_max_err(h, direct) < 1e-13


def test_o9_every_valid_tuple_tiny():
    n, L = 3, 6
    xs = synth.unit_disk(77, (n, L))
    want = first_L_iterated(xs)
    Mmin = n * (L - 1) + 1
    for m in range(1, 2 * Mmin):
        for p in (-(-L // m), -(-L // m) + 1):
            q = -(-Mmin // m)
            assert rel_max_err(oracle.conv_multi(xs, m, p, q), want) < 1e-13, (m, p, q)


def test_o9_exact_integers():
    n, L = 4, 200
    parts = [synth.small_ints(900 + i, (L,)) for i in range(n)]
    xs = np.array([re + 1j * im for re, im in parts])
    re, im = parts[0]
    for re2, im2 in parts[1:]:
        re, im = oracle.conv_int_exact(re, im, re2, im2, method="direct")
    for m in (64, 128, 801):
        h = oracle.conv_multi(xs, m)
        assert np.array_equal(np.rint(h.real).astype(np.int64), re), m
        assert np.array_equal(np.rint(h.imag).astype(np.int64), im), m


def test_o9_closed_form_equal_ratio():
    L = 64
    a = 0.97 * np.exp(0.3j)
    for n in (2, 3, 5):
        xs = np.array([a ** np.arange(L)] * n)
        want = np.array([comb(k + n - 1, n - 1) * a ** k for k in range(L)])
        for m in (16, 48, 320):
            assert rel_max_err(oracle.conv_multi(xs, m), want) < 1e-13, (n, m)


def test_o9_reduces_to_o5_and_identity():
    L = 20
    xs = synth.unit_disk(88, (2, L))
    for m, p, q in ((8, 3, 5), (40, 1, 1), (5, 4, 8)):
        assert rel_max_err(oracle.conv_multi(xs, m, p, q), oracle.conv_hybrid(xs[0], xs[1], m, p, q)) < 1e-14
    x1 = synth.unit_disk(89, (1, L))
    assert rel_max_err(oracle.conv_multi(x1, 8), x1[0]) < 1e-14


def test_o9_aliasing():
    n, L = 3, 10
    xs = synth.unit_disk(90, (n, L))
    # the alias-free minimum for n = 3, L = 10 is q m = 28
    oracle.conv_multi(xs, 4, 3, 7)
    with pytest.raises(RuntimeError):
        oracle.conv_multi(xs, 4, 3, 6)
    with pytest.raises(RuntimeError):
        oracle.conv_multi(xs, 19, 1, 1)     # 2 L - 1 = 19


def pairwise_sum(xs):
    L = xs.shape[1]
    return sum(np.convolve(xs[i], xs[i + 1])[:L] for i in range(0, xs.shape[0], 2))


@pytest.mark.parametrize("n,L,m", [(2, 9, 6), (4, 10, 4), (4, 10, 19), (6, 7, 5), (8, 33, 16), (4, 1, 1)])
def test_o9_dot_against_library_and_direct(n, L, m):
    xs = synth.unit_disk(800 + 10 * n + L, (n, L))
    h = oracle.conv_multi(xs, m, op="dot")
    assert rel_max_err(h, pairwise_sum(xs)) < 1e-13
    direct = sum(oracle.conv_direct(xs[i], xs[i + 1]) for i in range(0, n, 2))
    assert rel_max_err(h, direct) < 1e-13


def test_o9_dot_exact_integers_and_aliasing():
    n, L = 6, 300
    parts = [synth.small_ints(950 + i, (L,)) for i in range(n)]
    re = np.zeros(L, dtype=np.int64)
    im = np.zeros(L, dtype=np.int64)
    for i in range(0, n, 2):
        a, b = oracle.conv_int_exact(*parts[i], *parts[i + 1])
        re += a
        im += b
    xs = np.array([r + 1j * i for r, i in parts])
    for m in (64, 599, 128):
        h = oracle.conv_multi(xs, m, op="dot")
        assert np.array_equal(np.rint(h.real).astype(np.int64), re), m
        assert np.array_equal(np.rint(h.imag).astype(np.int64), im), m
    # 2 L - 1 suffices for the pairwise sum, one less does not; odd n is invalid
    oracle.conv_multi(xs, 599, 1, 1, op="dot")
    with pytest.raises(RuntimeError):
        oracle.conv_multi(xs, 598, 1, 1, op="dot")
    with pytest.raises(RuntimeError):
        oracle.conv_multi(xs[:5], 599, op="dot")

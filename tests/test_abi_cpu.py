"""Host-side checks of the C ABI: the library builds and loads, exports every
entry point include/hdc.h declares, and its parameter logic (Section 2.5,
Section 3.1) is right.  No GPU and no compute calls."""
import json
import os
import re

import pytest

import paper_2306_10016_gb300 as hdc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lib():
    hdc.build()
    return hdc.lib()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(hdc_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert "hdc_conv1d" in names and "hdc_strerror" in names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_header():
    declared = _declared_functions()
    bound = {n for n, _, _ in hdc._SIGS}
    assert declared <= bound | {n for n in declared if n.startswith("hdc_plan") or n.startswith("hdc_tune")}


def test_paper_parameter_example(lib):
    """Section 2.5, figure caption: L=6, M=11, m=4 => p=2, q=3."""
    with open(os.path.join(GOLD, "paper_1d_parameter_example.json")) as fh:
        ex = json.load(fh)
    p, q = hdc.derive_params(ex["L"], ex["M"], ex["m"])
    assert (p, q) == (ex["p"], ex["q"])
    assert p * ex["m"] == ex["explicit_pad_pm"] and q * ex["m"] == ex["implicit_pad_qm"]


def test_derive_params_smallest(lib):
    for L in range(1, 40):
        for M in range(L, 3 * L):
            for m in range(1, M + 2):
                p, q = hdc.derive_params(L, M, m)
                assert p * m >= L and (p - 1) * m < L
                assert q * m >= M and (q - 1) * m < M


def test_good_sizes(lib):
    def brute(n):
        for f in (2, 3, 5, 7):
            while n % f == 0:
                n //= f
        return n == 1
    for n in range(1, 3000):
        assert hdc.is_good_size(n) == brute(n)
    for n in [1, 2, 11, 13, 2047, 4095, 4097, 1023, 9999]:
        k = hdc.next_good_size(n)
        assert k >= n and brute(k) and all(not brute(j) for j in range(n, k))
    assert hdc.next_good_size(2047) == 2048
    assert hdc.next_good_size(11) == 12


def test_explicit_params(lib):
    assert hdc.explicit_params(1024, 2047) == (2048, 1, 1)
    assert hdc.explicit_params(6, 11) == (12, 1, 1)


def test_validation_errors(lib):
    C128 = hdc.HDC_C128
    # the L=1024, m=512 workload written with p=1 violates p m >= L (Section 2.5)
    rc, _ = hdc.validate_axis(1024, 2047, 512, 1, 4, 1, C128)
    assert rc == hdc.HDC_ERR_PARAM
    rc, (p, q, D) = hdc.validate_axis(1024, 2047, 512, 0, 0, 1, C128)
    assert rc == hdc.HDC_OK and (p, q, D) == (2, 4, 1)
    # alias: M < 2L-1
    assert hdc.validate_axis(1024, 2046, 512)[0] == hdc.HDC_ERR_ALIAS
    # m not 7-smooth
    assert hdc.validate_axis(100, 199, 11)[0] == hdc.HDC_ERR_UNSUPPORTED_SIZE
    # D > q
    assert hdc.validate_axis(100, 199, 50, 0, 0, 5)[0] == hdc.HDC_ERR_PARAM
    # q too small
    assert hdc.validate_axis(100, 199, 50, 2, 3)[0] == hdc.HDC_ERR_PARAM
    # bad dtype
    assert hdc.validate_axis(100, 199, 50, 0, 0, 0, 7)[0] == hdc.HDC_ERR_DTYPE
    # m beyond the limit
    big = hdc.max_fft_size(C128) * 2
    assert hdc.validate_axis(big, 2 * big, big)[0] == hdc.HDC_ERR_UNSUPPORTED_SIZE
    # every status has text
    for code in range(0, -10, -1):
        assert hdc.strerror(code) != "unknown status"


def test_workspace_size_monotone(lib):
    a = hdc.workspace_size([1024], [2047], [512], D=[1])
    b = hdc.workspace_size([1024], [2047], [512], D=[4])
    assert 0 < a < b
    c = hdc.workspace_size([64, 64], [127, 127], [64, 64])
    assert c > 0
    d = hdc.workspace_size([1 << 20], [(1 << 21) - 1], [1 << 20])
    assert d > 16 * (1 << 20)


def test_conv_rejects_before_launch(lib):
    """Bad arguments come back as codes from the host checks; no kernel runs
    (NULL pointers are never dereferenced)."""
    L = _ = 1024
    rc = lib.hdc_conv1d(None, None, None, 1024, 2047, 512, 1, 4, 1, 0, hdc.HDC_C128, 1, None, 0, None)
    assert rc == hdc.HDC_ERR_PARAM
    rc = lib.hdc_conv1d(None, None, None, 1024, 2047, 512, 0, 0, 1, 0, hdc.HDC_C128, 1, None, 0, None)
    assert rc == hdc.HDC_ERR_PARAM
    rc = lib.hdc_conv1d(None, None, None, 1024, 2047, 512, 0, 0, 1, 0, hdc.HDC_C128, 0, None, 0, None)
    assert rc == hdc.HDC_OK  # empty batch: nothing to do

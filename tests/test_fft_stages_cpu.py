"""The stage plans of the shared-memory FFTs (host only, through the C ABI):
the radices multiply to n, follow the stated order, take radix 16 exactly
where the rule says (complex<float> columns at any size, complex<float>
residue rows from 4096 points, never complex<double> or the other kernels),
and then use the fewest stages that radix 16 or 8 allows; errors for sizes
and arguments the kernels do not take."""
import ctypes as C
import math

import pytest

import paper_2306_10016_gb300 as hdc

F32, F64 = hdc.HDC_C64, hdc.HDC_C128
ROWS, COLS, OTHER = hdc.FFT_ROWS, hdc.FFT_COLS, hdc.FFT_OTHER


def _good(n):
    for f in (2, 3, 5, 7):
        while n % f == 0:
            n //= f
    return n == 1


def _e2(n):
    return (n & -n).bit_length() - 1


def _expected(n, r16):
    """Brute-force restatement of the rule: radix 16 while it divides the
    rest, when allowed and ceil(e/4) < ceil(e/3); then 8, 4, 2, 7, 5, 3."""
    rad, k = [], n
    e = _e2(n)
    if r16 and -(-e // 4) < -(-e // 3):
        while k % 16 == 0:
            rad.append(16)
            k //= 16
    for r in (8, 4, 2, 7, 5, 3):
        while k % r == 0:
            rad.append(r)
            k //= r
    assert k == 1
    return rad


@pytest.mark.parametrize("dtype", [F32, F64])
@pytest.mark.parametrize("kind", [ROWS, COLS, OTHER])
def test_stage_plans_over_all_good_sizes(dtype, kind):
    lim = hdc.lib().hdc_max_outer_fft_size(dtype) if kind == COLS else (2048 if dtype == F64 else 4096)
    for n in range(1, lim + 1):
        if not _good(n):
            continue
        rad = hdc.fft_stages(n, dtype, kind)
        assert math.prod(rad) == n
        r16 = dtype == F32 and (kind == COLS or (kind == ROWS and n >= 4096))
        assert rad == _expected(n, r16), n
        if 16 in rad:
            # radix 16 only where it saves a stage over radix 8
            assert len(rad) < len(_expected(n, False))


def test_named_plans():
    assert hdc.fft_stages(4096, F32, ROWS) == [16, 16, 16]
    assert hdc.fft_stages(2048, F32, ROWS) == [8, 8, 8, 4]        # rows below 4096: radix 8
    assert hdc.fft_stages(2048, F32, COLS) == [16, 16, 8]
    assert hdc.fft_stages(512, F32, COLS) == [8, 8, 8]             # 16 saves no stage
    assert hdc.fft_stages(256, F32, COLS) == [16, 16]
    assert hdc.fft_stages(48, F32, COLS) == [16, 3]
    assert hdc.fft_stages(4096, F32, OTHER) == [8, 8, 8, 8]
    assert hdc.fft_stages(2048, F64, ROWS) == [8, 8, 8, 4]
    assert hdc.fft_stages(4096, F64, COLS) == [8, 8, 8, 8]
    assert hdc.fft_stages(2800, F32, ROWS) == [8, 2, 7, 5, 5]
    assert hdc.fft_stages(1400, F64, ROWS) == [8, 7, 5, 5]
    assert hdc.fft_stages(1, F64, ROWS) == []


def test_errors():
    lib = hdc.lib()
    buf = (C.c_int * 32)()
    assert lib.hdc_fft_stages(4096, F64, ROWS, buf, 32) == hdc.HDC_ERR_UNSUPPORTED_SIZE  # above FP64 rows
    assert lib.hdc_fft_stages(8192, F32, ROWS, buf, 32) == hdc.HDC_ERR_UNSUPPORTED_SIZE
    assert lib.hdc_fft_stages(8192, F32, COLS, buf, 32) == 4                              # 16, 16, 16, 2
    assert lib.hdc_fft_stages(11, F32, COLS, buf, 32) == hdc.HDC_ERR_UNSUPPORTED_SIZE
    assert lib.hdc_fft_stages(0, F32, COLS, buf, 32) == hdc.HDC_ERR_UNSUPPORTED_SIZE
    assert lib.hdc_fft_stages(64, 7, COLS, buf, 32) == hdc.HDC_ERR_DTYPE
    assert lib.hdc_fft_stages(64, F32, 3, buf, 32) == hdc.HDC_ERR_PARAM
    assert lib.hdc_fft_stages(64, F32, COLS, None, 32) == hdc.HDC_ERR_PARAM
    assert lib.hdc_fft_stages(4096, F32, ROWS, buf, 2) == hdc.HDC_ERR_PARAM              # three stages

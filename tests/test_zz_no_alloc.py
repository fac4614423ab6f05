"""The allocation-free 1-D entry point (hdc_conv1d_noalloc), called through
the C ABI, against the regular entry point (hdc_conv1d) on the same inputs.

hdc_conv1d_noalloc exists for callers that cannot allocate device memory
while they run (a plugin inside an application that owns the device-memory
budget, a real-time loop that cannot take cudaMalloc's synchronisation): its
scratch is a fixed device array inside the library.  This file is collected
last so a stop at the first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2306_10016_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 5e-5}


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_10016_gb300 as h
    h.build()
    h.lib()
    return h


def _rel(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _noalloc_abi(hdc, f, g, h, L, m, D):
    st = torch.cuda.current_stream()
    return hdc.lib().hdc_conv1d_noalloc(C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()),
                                        C.c_void_p(h.data_ptr()), L, 2 * L - 1, m, 0, 0, D,
                                        hdc.dtype_code(f.dtype), f.numel() // L, C.c_void_p(st.cuda_stream))


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64])
def test_noalloc_matches_conv1d_two_calls(hdc, dt):
    # two calls in a row with different problems: the second must not see
    # anything the first left in the shared scratch array
    cases = [(3, 3000, 1024, 2), (2, 1000, 250, 0)]
    for k, (B, L, m, D) in enumerate(cases):
        f = torch.from_numpy(synth.unit_disk(900 + k, (B, L))).to("cuda", dt)
        g = torch.from_numpy(synth.unit_disk(950 + k, (B, L))).to("cuda", dt)
        ref = hdc.conv1d(f, g, m, D=D)
        h = torch.full_like(f, complex("nan+nanj"))
        assert _noalloc_abi(hdc, f, g, h, L, m, D) == hdc.HDC_OK
        torch.cuda.synchronize()
        assert _rel(h, ref) <= TOL[dt], (dt, B, L, m, D)


def test_noalloc_rejects_oversize_and_aliasing(hdc):
    L, m = 20000, 8192
    f = torch.zeros((L,), dtype=torch.complex128, device="cuda")
    g = torch.zeros_like(f)
    h = torch.empty_like(f)
    # m beyond the single-tile route (FP64: 2048)
    assert _noalloc_abi(hdc, f, g, h, L, m, 0) == hdc.HDC_ERR_UNSUPPORTED_SIZE
    # workspace beyond the fixed scratch array: 64 rows x q=16 x 2048 x 16 B = 32 MiB + tables
    B, L, m = 64, 16384, 2048
    f = torch.zeros((B, L), dtype=torch.complex128, device="cuda")
    g = torch.zeros_like(f)
    h = torch.empty_like(f)
    assert _noalloc_abi(hdc, f, g, h, L, m, 0) == hdc.HDC_ERR_UNSUPPORTED_SIZE
    # h aliasing an input
    assert _noalloc_abi(hdc, f, g, f, L, m, 1) == hdc.HDC_ERR_PARAM

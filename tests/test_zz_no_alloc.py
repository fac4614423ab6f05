"""The allocation-free 1-D entry point (hdc_conv1d_noalloc), called through
the C ABI, against the CPU oracle and against the regular entry point
(hdc_conv1d, also through the C ABI) on the same inputs.

hdc_conv1d_noalloc exists for callers that cannot allocate device memory
while they run (a plugin inside an application that owns the device-memory
budget, a real-time loop that cannot take cudaMalloc's synchronisation): its
scratch is a fixed device array inside the library.  This file is collected
last so a stop at the first failure has run every other test; every test
here also passes on its own in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import oracle
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


def _rel(a, ref):
    a = a.cpu().numpy().astype(np.complex128)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def _noalloc_abi(hdc, f, g, h, L, m, D, p=0, q=0):
    st = torch.cuda.current_stream()
    return hdc.lib().hdc_conv1d_noalloc(C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()),
                                        C.c_void_p(h.data_ptr()), L, 2 * L - 1, m, p, q, D,
                                        hdc.dtype_code(f.dtype), f.numel() // L, C.c_void_p(st.cuda_stream))


def _conv1d_abi(hdc, f, g, h, L, m, D, p=0, q=0):
    """The regular entry point with a workspace allocated here by torch."""
    dt = hdc.dtype_code(f.dtype)
    B = f.numel() // L
    nb = hdc.workspace_size([L], [2 * L - 1], [m], p=[p], q=[q], D=[D], dtype=dt, batch=B)
    ws = torch.empty(max(1, nb), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    hdc.prepare([L], [m], p=[p], q=[q], D=[D], dtype=dt, batch=B)
    rc = hdc.lib().hdc_conv1d(C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), C.c_void_p(h.data_ptr()),
                              L, 2 * L - 1, m, p, q, D, 0, dt, B, C.c_void_p(ws.data_ptr()), C.c_size_t(nb),
                              C.c_void_p(st.cuda_stream))
    torch.cuda.synchronize()
    return rc


def _oracle_rows(f, g):
    """Eq. 4 per row: the direct sum (O1) for short rows, the explicitly
    padded FFT convolution (O2) for long ones."""
    conv = oracle.conv_direct if f.shape[1] <= 4096 else oracle.conv_fft
    return np.stack([conv(f[b], g[b]) for b in range(f.shape[0])])


# (batch, L, m, D, p): several residue passes (D < q), a partial last pass,
# all residues at once, an explicit p above ceil(L / m), explicit padding
# (q = 1), and an FP32-relevant N = q m above 2^16 (L = 40000, m = 4096:
# q = 20, N = 81920)
CASES = [(3, 3000, 1024, 2, 0), (2, 1000, 250, 0, 0), (1, 2000, 512, 3, 6), (2, 700, 1400, 0, 0),
         (1, 40000, 4096, 4, 0)]


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64])
def test_noalloc_matches_oracle_and_conv1d(hdc, dt):
    # calls in a row with different problems: none may see anything an
    # earlier one left in the shared scratch array
    for k, (B, L, m, D, p) in enumerate(CASES):
        if dt == torch.complex128 and m > 2048:    # the FP64 single-tile route ends at 2048
            continue
        fn = synth.unit_disk(900 + k, (B, L))
        gn = synth.unit_disk(950 + k, (B, L))
        ref = _oracle_rows(fn, gn)
        f = torch.from_numpy(fn).to("cuda", dt)
        g = torch.from_numpy(gn).to("cuda", dt)
        h = torch.full_like(f, complex("nan+nanj"))
        assert _noalloc_abi(hdc, f, g, h, L, m, D, p=p) == hdc.HDC_OK
        torch.cuda.synchronize()
        err = _rel(h, ref)
        assert err <= TOL[dt], (dt, B, L, m, D, p, err)
        # and the regular entry point on the same inputs
        h2 = torch.full_like(f, complex("nan+nanj"))
        assert _conv1d_abi(hdc, f, g, h2, L, m, D, p=p) == hdc.HDC_OK
        assert _rel(h, h2.cpu().numpy().astype(np.complex128)) <= TOL[dt], (dt, B, L, m, D, p)


def test_noalloc_exact_integers_fp64(hdc):
    # integer inputs in [-8, 8]: the FP64 result rounds to the exact integer
    # convolution (oracle O3), twice in a row
    for k, (L, m, D) in enumerate([(1500, 512, 1), (4096, 2048, 0)]):
        fre, fim = synth.small_ints(700 + k, (L,))
        gre, gim = synth.small_ints(750 + k, (L,))
        hre, him = oracle.conv_int_exact(fre, fim, gre, gim)
        f = torch.from_numpy(synth.ints_to_complex(fre, fim)).to("cuda")
        g = torch.from_numpy(synth.ints_to_complex(gre, gim)).to("cuda")
        h = torch.full_like(f, complex("nan+nanj"))
        assert _noalloc_abi(hdc, f, g, h, L, m, D) == hdc.HDC_OK
        torch.cuda.synchronize()
        out = h.cpu().numpy()
        assert np.array_equal(np.rint(out.real).astype(np.int64), hre)
        assert np.array_equal(np.rint(out.imag).astype(np.int64), him)


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

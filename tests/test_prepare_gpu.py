"""The convolution calls allocate nothing: their twiddle tables come from the
preparation calls (hdc_prepare*, hdc_plan_create).  Through the C ABI:

* a call whose tables were never made returns HDC_ERR_NOT_PREPARED and
  leaves its output untouched;
* after hdc_plan_create, the plan's very first hdc_plan_execute can be
  captured in a CUDA graph (no allocation or synchronisation inside it) and
  its replays match the oracle's explicitly padded FFT convolution (O2),
  on the single-tile route and on a split transform, in both dtypes.

The sizes here (m = 1134 and 6174) are used by no other test, so their
tables are made in this file for the first time."""
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


def _a(*v):
    return (C.c_int64 * len(v))(*v)


def test_unprepared_call_is_refused(hdc):
    L, m = 1900, 1134            # q = ceil(3799 / 1134) = 4, N = 4536
    f = torch.from_numpy(synth.unit_disk(11, (L,))).to("cuda")
    g = torch.from_numpy(synth.unit_disk(12, (L,))).to("cuda")
    h = torch.full_like(f, complex("nan+nanj"))
    nb = hdc.workspace_size([L], [2 * L - 1], [m])
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    rc = hdc.lib().hdc_conv1d(C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), C.c_void_p(h.data_ptr()),
                              L, 2 * L - 1, m, 0, 0, 0, 0, hdc.HDC_C128, 1, C.c_void_p(ws.data_ptr()),
                              C.c_size_t(nb), C.c_void_p(st.cuda_stream))
    assert rc == hdc.HDC_ERR_NOT_PREPARED
    torch.cuda.synchronize()
    assert torch.isnan(h.real).all()
    # prepared, the same call runs and matches the oracle
    assert hdc.lib().hdc_prepare(1, _a(L), _a(2 * L - 1), _a(m), None, None, None, hdc.HDC_C128, 1) == hdc.HDC_OK
    rc = hdc.lib().hdc_conv1d(C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()), C.c_void_p(h.data_ptr()),
                              L, 2 * L - 1, m, 0, 0, 0, 0, hdc.HDC_C128, 1, C.c_void_p(ws.data_ptr()),
                              C.c_size_t(nb), C.c_void_p(st.cuda_stream))
    assert rc == hdc.HDC_OK
    torch.cuda.synchronize()
    ref = oracle.conv_fft(f.cpu().numpy(), g.cpu().numpy())
    assert np.max(np.abs(h.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-12


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("L,m,B", [(2000, 1134, 3), (6000, 6174, 1)])
def test_first_plan_execute_captured_in_graph(hdc, dt, L, m, B):
    code = hdc.dtype_code(dt)
    plan = C.c_void_p()
    assert hdc.lib().hdc_plan_create(C.byref(plan), 1, _a(L), _a(2 * L - 1), _a(m), None, code, B,
                                     hdc.HDC_FIXED, None, None) == hdc.HDC_OK
    try:
        fn = synth.unit_disk(21 + m, (B, L))
        gn = synth.unit_disk(22 + m, (B, L))
        f = torch.from_numpy(fn).to("cuda", dt)
        g = torch.from_numpy(gn).to("cuda", dt)
        h = torch.full_like(f, complex("nan+nanj"))
        nb = hdc.lib().hdc_plan_workspace(plan)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        rcs = []
        with torch.cuda.graph(graph, stream=side):
            rcs.append(hdc.lib().hdc_plan_execute(plan, C.c_void_p(f.data_ptr()), C.c_void_p(g.data_ptr()),
                                                  C.c_void_p(h.data_ptr()), C.c_void_p(ws.data_ptr()),
                                                  C.c_size_t(nb), C.c_void_p(side.cuda_stream)))
        assert rcs == [hdc.HDC_OK]
        for _ in range(2):
            h.fill_(complex("nan+nanj"))
            graph.replay()
            torch.cuda.synchronize()
            out = h.cpu().numpy().astype(np.complex128)
            for b in range(B):
                ref = oracle.conv_fft(fn[b], gn[b])
                err = np.max(np.abs(out[b] - ref)) / np.max(np.abs(ref))
                assert err <= TOL[dt], (dt, L, m, b, err)
        del graph
    finally:
        hdc.lib().hdc_plan_destroy(plan)

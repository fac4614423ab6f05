"""Output windows of the linear convolution and the centered Hermitian 2-D
convolution (padding ratio 3/2) on the GPU, against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_10016_gb300 as h
    h.build()
    h.lib()
    return h


def _full_linear(f, g):
    """Whole linear convolution from the oracle: zero-pad both inputs to
    2L-1 per axis; the first 2L-1 outputs of that are the full convolution."""
    pad = [(0, n - 1) for n in f.shape]
    return oracle.conv_direct(np.pad(f, pad), np.pad(g, pad))


@pytest.mark.parametrize("L,m,D", [(100, 64, 0), (1000, 500, 1), (777, 2000, 0), (3000, 7000, 0), (5000, 1000, 2)])
def test_full_length_1d(hdc, L, m, D):
    f = synth.unit_disk(301, (L,))
    g = synth.unit_disk(302, (L,))
    ref = _full_linear(f, g)
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    h = hdc.convnd_window(ft, gt, 1, m, o=0, Lw=2 * L - 1, D=D)
    torch.cuda.synchronize()
    assert rel_max_err(h.cpu().numpy(), ref) < 1e-12


def test_middle_window_less_padding(hdc):
    L = 600
    f = synth.unit_disk(303, (L,))
    g = synth.unit_disk(304, (L,))
    ref = _full_linear(f, g)
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    o, Lw = 300, 500
    M = 2 * L - 1 - o                      # the least padding that keeps [o, o+Lw) alias-free
    h = hdc.convnd_window(ft, gt, 1, 250, o=o, Lw=Lw, M=M)
    torch.cuda.synchronize()
    assert rel_max_err(h.cpu().numpy(), ref[o:o + Lw]) < 1e-12
    with pytest.raises(hdc.HDCError) as ei:     # one less is rejected
        hdc.convnd_window(ft, gt, 1, 250, o=o, Lw=Lw, M=M - 1)
    assert ei.value.code == hdc.HDC_ERR_ALIAS


@pytest.mark.parametrize("dt,tol", [(torch.complex128, 1e-12), (torch.complex64, 5e-5)])
def test_window_2d(hdc, dt, tol):
    shape = (30, 41)
    f = synth.unit_disk(305, shape)
    g = synth.unit_disk(306, shape)
    ref = _full_linear(f, g)
    ft = torch.from_numpy(f).to("cuda", dt)
    gt = torch.from_numpy(g).to("cuda", dt)
    h = hdc.convnd_window(ft, gt, 2, [16, 40], o=[10, 0], Lw=[45, 81])
    torch.cuda.synchronize()
    assert rel_max_err(h.cpu().numpy(), ref[10:55, 0:81]) < tol


@pytest.mark.parametrize("K,m", [(1, None), (2, None), (4, None), (8, [4, 16]), (17, [18, 9]), (33, [16, 35])])
def test_hermitian_small_vs_direct(hdc, K, m):
    f = synth.hermitian_normal(400 + K, K)
    g = synth.hermitian_normal(500 + K, K)
    ref = oracle.conv_hermitian_direct(f, g)
    h = hdc.conv2d_hermitian(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), m=m)
    torch.cuda.synchronize()
    assert rel_max_err(h.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("K,dt,tol", [(128, torch.complex128, 1e-12), (128, torch.complex64, 5e-5),
                                      (512, torch.complex128, 1e-12), (512, torch.complex64, 5e-5)])
def test_hermitian_vs_fft_oracle(hdc, K, dt, tol):
    """K = 512: the 1024 x 1024 real-field configuration (padding 1536 per axis)."""
    f = synth.hermitian_normal(600 + K, K)
    g = synth.hermitian_normal(700 + K, K)
    ref = oracle.conv_hermitian_fft(f, g)
    h = hdc.conv2d_hermitian(torch.from_numpy(f).to("cuda", dt), torch.from_numpy(g).to("cuda", dt))
    torch.cuda.synchronize()
    hn = h.cpu().numpy().astype(np.complex128)
    assert rel_max_err(hn, ref) < tol
    c = K - 1
    # the product of two real fields is real: the ky = 0 column is conjugate-symmetric
    assert np.max(np.abs(hn[::-1, 0] - np.conj(hn[:, 0]))) < 10 * tol * np.max(np.abs(ref))


def test_hermitian_batch(hdc):
    K, B = 16, 3
    f = np.stack([synth.hermitian_normal(800 + b, K) for b in range(B)])
    g = np.stack([synth.hermitian_normal(900 + b, K) for b in range(B)])
    h = hdc.conv2d_hermitian(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), m=[8, 8], D=[1, 2])
    torch.cuda.synchronize()
    for b in range(B):
        assert rel_max_err(h[b].cpu().numpy(), oracle.conv_hermitian_direct(f[b], g[b])) < 1e-12

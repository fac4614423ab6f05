"""FP32 transforms with radix-16 stages against the oracle.

FP32 rows of 4096 points and FP32 column transforms whose power-of-two part
saves a stage with radix 16 (16, 48 = 16 x 3, 112 = 16 x 7, 128, 256, 768,
2048 points, ...) run kernels built with a 16-point butterfly, whose twiddles
are products of four table entries; rows below 4096 points and the other
column sizes keep radix 8.  The cases mix both kinds of kernel in one
convolution (rows with and columns without radix 16, and the reverse), in
1-D, batched and 2-D/3-D, forward and inverse, at several residues per
pass."""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 5e-5


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2306_10016_gb300 as h
    h.build()
    h.lib()
    return h


def _pair(shape, seed):
    f = synth.unit_disk(seed, shape)
    g = synth.unit_disk(seed + 1, shape)
    return f, g, torch.from_numpy(f).to("cuda", torch.complex64), torch.from_numpy(g).to("cuda", torch.complex64)


@pytest.mark.parametrize("shape,m,D", [
    ((3000,), 4096, 1),           # fused rows of 4096 (16, 16, 16), q = 2
    ((4000,), 8192, 0),           # m = 2 x 4096
    ((8, 120000), 196608, 2),     # columns of 48 (16, 3) under rows of 4096, q = 2
    ((8, 200000), 458752, 0),     # columns of 112 (16, 7)
    ((4, 300000), 524288, 1),     # columns of 128 (16, 8), two passes
    ((8, 50000), 81920, 2),       # columns of 20 (radix-8 kernel), rows of 4096
    ((2, 600000), 1048576, 0),    # columns of 256 (16, 16)
    ((70001,), 131072, 1),        # 1-D, ragged tail
])
def test_conv1d_fp32_radix16(hdc, shape, m, D):
    f, g, ft, gt = _pair(shape, 8100 + shape[-1] % 89)
    h = hdc.conv1d(ft, gt, m, D=D).cpu().numpy()
    assert hdc.device_status() == 0
    if len(shape) == 1:
        assert rel_max_err(h, oracle.conv_fft(f, g)) < TOL32
    else:
        for i in range(shape[0]):
            assert rel_max_err(h[i], oracle.conv_fft(f[i], g[i])) < TOL32


@pytest.mark.parametrize("shape,m", [
    ((2048, 40), [4096, 96]),         # rows of 4096 along the outer axis
    ((100, 2100), [256, 4096]),       # last axis 4096 points, outer 256
    ((30, 40, 2000), [64, 80, 4096]),
])
def test_convnd_fp32_radix16(hdc, shape, m):
    f, g, ft, gt = _pair(shape, 8200 + len(shape))
    h = hdc.convnd(ft, gt, len(shape), m).cpu().numpy()
    assert hdc.device_status() == 0
    assert rel_max_err(h, oracle.conv_fft(f, g)) < TOL32


def test_radix16_fp32_matches_fp64(hdc):
    """The same 2^20-point convolution in FP32 (radix-16 rows and columns)
    and FP64 (radix 8): agreement within the FP32 bound, so the FP32 result
    is not merely self-consistent."""
    L, m = 600000, 1048576
    f, g, ft, gt = _pair((L,), 8300)
    h32 = hdc.conv1d(ft, gt, m).cpu().numpy()
    h64 = hdc.conv1d(ft.to(torch.complex128), gt.to(torch.complex128), m).cpu().numpy()
    assert rel_max_err(h32, h64) < TOL32
    assert np.isfinite(h32).all()

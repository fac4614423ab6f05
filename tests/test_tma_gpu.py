"""The strided fold's two load paths: tiles staged by TMA box copies and the
plain loads.  Both fold the same values in the same order: in FP64 their
outputs are bit-identical; in FP32, whose large fold twiddles are products of
two table entries formed inside each kernel, they agree to rounding.  The
cases cover partial last rows, one and two fold blocks, several boxes per
block, batches, 2-D/3-D outer axes, several inputs per launch, and layouts
that must fall back to the plain loads."""
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
    yield h
    h.set_tma(True)


def _both(hdc, run):
    """run() on plain loads, then with TMA allowed; returns both outputs and
    the number of TMA-staged fold launches of the second run.  The
    thread-block-cluster route (which has no strided fold) is turned off, so
    short single rows take the split route whose fold this file tests."""
    hdc.set_cluster(0)
    try:
        hdc.set_tma(False)
        a = run().cpu().numpy()
        hdc.set_tma(True)
        hdc.stats_reset()
        b = run().cpu().numpy()
        torch.cuda.synchronize()
        n_tma = hdc.stats()["k_fold_fft_cols_tma"]["launches"]
    finally:
        hdc.set_cluster(1)
    assert hdc.device_status() == 0
    return a, b, n_tma


def _same(a, b):
    """Bit-identical in FP64; within 2e-6 of the larger magnitude in FP32."""
    if a.dtype in (np.complex128, np.float64):
        return np.array_equal(a, b)
    return float(np.max(np.abs(a - b))) <= 2e-6 * float(np.max(np.abs(a)))


def _inputs(shape, seed, dt):
    f = synth.unit_disk(seed, shape)
    g = synth.unit_disk(seed + 1, shape)
    return f, g, torch.from_numpy(f).to("cuda", dt), torch.from_numpy(g).to("cuda", dt)


DT = [(torch.complex128, 1e-12), (torch.complex64, 5e-5)]


@pytest.mark.parametrize("dt,tol", DT)
@pytest.mark.parametrize("L,m,D", [
    (40000, 32768, 1),    # p = 2, q = 3, partial last row, second block past the full rows
    (40000, 32768, 3),    # all residues in one pass
    (5000, 16384, 1),     # explicit (p = q = 1), partial row
    (98304, 65536, 2),    # L a multiple of the row length
    (458753, 917504, 0),  # FP64 ma = 448: two boxes of 224 rows
    (786433, 1572864, 0),  # FP64 ma = 768: three boxes of 256 rows
])
def test_split_1d_tma_matches_plain(hdc, dt, tol, L, m, D):
    f, g, ft, gt = _inputs((L,), 7100 + L % 97, dt)
    a, b, n_tma = _both(hdc, lambda: hdc.conv1d(ft, gt, m, D=D))
    assert n_tma > 0
    assert _same(a, b)
    assert rel_max_err(b, oracle.conv_fft(f, g)) < tol


@pytest.mark.parametrize("dt,tol", DT)
def test_batched_rows_tma_matches_plain(hdc, dt, tol):
    f, g, ft, gt = _inputs((3, 20000), 7200, dt)
    a, b, n_tma = _both(hdc, lambda: hdc.conv1d(ft, gt, 16384, D=2))
    assert n_tma > 0 and _same(a, b)
    for i in range(3):
        assert rel_max_err(b[i], oracle.conv_fft(f[i], g[i])) < tol


@pytest.mark.parametrize("dt,tol", DT)
@pytest.mark.parametrize("shape,m", [((300, 200), [512, 400]), ((40, 48, 56), [80, 96, 112]),
                                     ((700, 64), [1024, 128])])
def test_outer_axes_tma_matches_plain(hdc, dt, tol, shape, m):
    f, g, ft, gt = _inputs(shape, 7300 + len(shape), dt)
    a, b, n_tma = _both(hdc, lambda: hdc.convnd(ft, gt, len(shape), m))
    assert n_tma > 0 and _same(a, b)
    assert rel_max_err(b, oracle.conv_fft(f, g)) < tol


def test_odd_row_length_falls_back(hdc):
    """FP32 rows of an odd number of complex values are not 16-byte strided:
    the fold takes the plain loads (and the result is the same)."""
    f, g, ft, gt = _inputs((60, 201), 7400, torch.complex64)
    a, b, n_tma = _both(hdc, lambda: hdc.convnd(ft, gt, 2, [128, 405]))
    assert n_tma == 0 and _same(a, b)
    assert rel_max_err(b, oracle.conv_fft(f, g)) < 5e-5


def test_multi_and_real_tma_match_plain(hdc):
    xs_np = [synth.unit_disk(7500 + i, (30000,)) for i in range(4)]
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    a, b, n_tma = _both(hdc, lambda: hdc.convnd_multi(xs, 1, [16384], op="dot"))
    assert n_tma > 0 and _same(a, b)
    fr = torch.from_numpy(synth.standard_normal(7510, 30000)).cuda()
    gr = torch.from_numpy(synth.standard_normal(7511, 30000)).cuda()
    a, b, n_tma = _both(hdc, lambda: hdc.convnd_real(fr, gr, 1, [16384]))
    assert n_tma > 0 and _same(a, b)


def test_first_launch_at_the_shared_memory_threshold(hdc):
    """A fresh process whose first TMA fold needs 48 KiB of dynamic shared
    memory (ma = 384, C = 4): with the barrier's static bytes that is past the
    default limit, so the launcher must opt the kernel in first (it used to
    fail with cudaErrorInvalidValue until a larger launch had done so)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import numpy as np, torch, oracle\n"
            "import paper_2306_10016_gb300 as hdc\n"
            "from paper_2306_10016_gb300 import synth\n"
            "f = synth.unit_disk(7600, (49152,)); g = synth.unit_disk(7601, (49152,))\n"
            "hdc.stats_reset()\n"
            "h = hdc.conv1d(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), 49152, D=2).cpu().numpy()\n"
            "assert hdc.stats()['k_fold_fft_cols_tma']['launches'] > 0\n"
            "ref = oracle.conv_fft(f, g)\n"
            "print(float(np.max(np.abs(h - ref)) / np.max(np.abs(ref))))\n")
    env = dict(os.environ, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert float(r.stdout.strip().splitlines()[-1]) < 1e-12

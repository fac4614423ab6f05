"""The thread-block-cluster route (k_conv_cluster): whole 1-D convolutions of
a few short rows in one launch, transforms spread over a cluster and
transposed through distributed shared memory.  Through the C ABI, against
the oracle (O1, O2; exact integers O3) and against the same calls with the
route turned off, in FP64 and FP32: several residues and fold blocks,
explicit and implicit padding, a batch of rows, an output window, residue
shares, and the largest residues the route takes."""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err

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
    yield h
    h.set_cluster(1)


def _conv(hdc, f, g, m, D=0, cluster=2, **kw):
    """The convolution with the cluster route forced on (any m whose factors
    fit a cluster) or off; returns it and the number of cluster launches."""
    hdc.set_cluster(cluster)
    hdc.stats_reset()
    h = hdc.conv1d(f, g, m, D=D, **kw)
    torch.cuda.synchronize()
    n = hdc.stats()["k_conv_cluster"]["launches"]
    hdc.set_cluster(1)
    return h.cpu().numpy().astype(np.complex128), n


CASES = [
    # (batch, L, m): L = 1024 with (m, p, q) = (512, 2, 4) and (256, 4, 8),
    # explicit padding, implicit q = 2, ragged L, and the largest residues
    (1, 1024, 512), (1, 1024, 256), (1, 1024, 2048), (1, 2048, 2048), (3, 3000, 1024), (2, 5000, 8192),
    (1, 16384, 16384), (1, 6000, 12288),
    # two points per lane in the shuffle transforms: 32 x 64 and 64 x 64
    (2, 1500, 2048), (2, 3000, 4096),
    # many residues and fold blocks on the shuffle path (q = 20, p = 10;
    # FP32 fold twiddles from the split table, N = 81920)
    (1, 40000, 4096),
]


@pytest.mark.parametrize("dt", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("B,L,m", CASES)
def test_cluster_route_against_oracle(hdc, dt, B, L, m):
    fn = synth.unit_disk(31000 + L, (B, L))
    gn = synth.unit_disk(32000 + L, (B, L))
    f = torch.from_numpy(fn).to("cuda", dt)
    g = torch.from_numpy(gn).to("cuda", dt)
    h, n = _conv(hdc, f, g, m)
    assert n == 1, "the cluster route was not taken"
    conv = oracle.conv_direct if L <= 4096 else oracle.conv_fft
    for b in range(B):
        ref = conv(fn[b], gn[b])
        assert rel_max_err(h[b], ref) <= TOL[dt], (B, L, m, b)
    h2, n2 = _conv(hdc, f, g, m, cluster=0)
    assert n2 == 0
    assert rel_max_err(h, h2) <= 2 * TOL[dt]


def test_cluster_route_exact_integers(hdc):
    for L, m in ((1024, 512), (4096, 8192)):
        fr, fi = synth.small_ints(33000 + L, (L,))
        gr, gi = synth.small_ints(34000 + L, (L,))
        hr, hi = oracle.conv_int_exact(fr, fi, gr, gi)
        f = torch.from_numpy(synth.ints_to_complex(fr, fi)).cuda()
        g = torch.from_numpy(synth.ints_to_complex(gr, gi)).cuda()
        h, n = _conv(hdc, f, g, m)
        assert n == 1
        assert np.array_equal(np.rint(h.real).astype(np.int64), hr)
        assert np.array_equal(np.rint(h.imag).astype(np.int64), hi)


@pytest.mark.parametrize("L,m", [(6000, 8192), (3000, 2048), (1000, 512)])
def test_cluster_route_window_and_residue_shares(hdc, L, m):
    """m = 8192: shared-memory transforms; m = 2048 and 512: the warp-shuffle
    ones (two points and one point per lane)."""
    fn = synth.unit_disk(35001, (L,))
    gn = synth.unit_disk(35002, (L,))
    f = torch.from_numpy(fn).cuda()
    g = torch.from_numpy(gn).cuda()
    full = oracle.conv_direct(np.concatenate([fn, np.zeros(L)]), np.concatenate([gn, np.zeros(L)]))[:2 * L - 1]
    hdc.set_cluster(2)
    try:
        hdc.stats_reset()
        lo, n = L // 3, L + L // 6
        hw = hdc.convnd_window(f, g, 1, m, lo, n).cpu().numpy()
        torch.cuda.synchronize()
        assert hdc.stats()["k_conv_cluster"]["launches"] == 1
        assert rel_max_err(hw, full[lo:lo + n]) <= 1e-12
        # the shares of disjoint residue ranges add up to the convolution
        q = -(-(2 * L - 1) // m)
        parts = [hdc.convnd_residues(f, g, 1, m, lo, hi) for lo, hi in ((0, 1), (1, q))]
        tot = (parts[0] + parts[1]).cpu().numpy()
        assert rel_max_err(tot, full[:L]) <= 1e-12
    finally:
        hdc.set_cluster(1)


def test_cluster_route_closed_form(hdc):
    L, P = 16384, (1 << 26) + 7
    f = torch.from_numpy(synth.exp_seq(12345, P, L)).cuda()
    g = torch.from_numpy(synth.exp_seq(67891, P, L)).cuda()
    h, n = _conv(hdc, f, g, 16384)
    assert n == 1
    assert rel_max_err(h, oracle.closed_form_exp(12345, 67891, P, L)) <= 1e-12

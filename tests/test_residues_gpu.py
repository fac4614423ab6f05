"""Residue-range shares (hdc_convnd_residues) on one GPU: disjoint ranges
add up to the convolution -- the computation each rank of a residue-sharded
multi-GPU convolution performs before the sum-reduction."""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import sharding, synth
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


@pytest.mark.parametrize("shape,m,D,world", [((3000,), 512, 2, 2), ((3000,), 512, 0, 3), ((20000,), 8192, 1, 2),
                                             ((48, 40), [16, 40], [2, 0], 2), ((9, 10, 11), [6, 20, 7], 0, 3)])
def test_shares_add_up(hdc, shape, m, D, world):
    f = synth.unit_disk(700, shape)
    g = synth.unit_disk(701, shape)
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    dims = len(shape)
    m0 = m[0] if isinstance(m, list) else m
    q0 = -(-(2 * shape[0] - 1) // m0)
    total = torch.zeros_like(ft)
    for lo, hi in sharding.residue_ranges(q0, world):
        if hi > lo:
            total += hdc.convnd_residues(ft, gt, dims, m, lo, hi, D=D)
    torch.cuda.synchronize()
    ref = oracle.conv_direct(f, g) if f.size <= 5000 else oracle.conv_fft(f, g)
    assert rel_max_err(total.cpu().numpy(), ref) < 1e-12
    full = hdc.convnd(ft, gt, dims, m, D=D)
    torch.cuda.synchronize()
    assert rel_max_err(total.cpu().numpy(), full.cpu().numpy()) < 1e-13


def test_bad_ranges_rejected(hdc):
    ft = torch.zeros((100,), dtype=torch.complex128, device="cuda")
    for lo, hi in ((2, 2), (-1, 1), (0, 5)):        # q = 4 for m = 50
        with pytest.raises(hdc.HDCError):
            hdc.convnd_residues(ft, ft.clone(), 1, 50, lo, hi)

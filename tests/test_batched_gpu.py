"""The batched persistent kernel: many convolutions of uneven length in one
cooperative launch, against the CPU oracle; CUDA-graph replay; the bounded
grid barrier's timeout path (no fault, no hang)."""
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


def _problem(n, lo, hi, seed, dt, extra=()):
    Ls = list(synth.log_uniform_lengths(seed, n, lo, hi)) + list(extra)
    fs = [synth.unit_disk(seed * 1000 + 2 * i, (int(L),)) for i, L in enumerate(Ls)]
    gs = [synth.unit_disk(seed * 1000 + 2 * i + 1, (int(L),)) for i, L in enumerate(Ls)]
    ft = [torch.from_numpy(f).to("cuda", dt) for f in fs]
    gt = [torch.from_numpy(g).to("cuda", dt) for g in gs]
    ht = [torch.empty_like(f) for f in ft]
    return [int(L) for L in Ls], fs, gs, ft, gt, ht


def _check(fs, gs, ht, tol):
    for f, g, h in zip(fs, gs, ht):
        ref = oracle.conv_direct(f, g) if f.size <= 6000 else oracle.conv_fft(f, g)
        assert rel_max_err(h.cpu().numpy(), ref) < tol, f.size


@pytest.mark.parametrize("dt,tol", [(torch.complex128, 1e-12), (torch.complex64, 5e-5)])
def test_batched_fixed_m(hdc, dt, tol):
    # explicit m for some, hybrid m for others; the extra lengths force the
    # split route (m above one row tile)
    Ls, fs, gs, ft, gt, ht = _problem(30, 64, 4096, 7, dt, extra=(20000, 9000))
    ms = []
    for i, L in enumerate(Ls):
        M = 2 * L - 1
        ms.append(hdc.next_good_size(M) if i % 2 else hdc.next_good_size((M + 3) // 4))
    dcode = hdc.dtype_code(dt)
    plan = hdc.BatchedPlan(Ls, ms, dcode)
    assert any(p["m1"] > 0 for p in plan.params) and any(p["m1"] == 0 for p in plan.params)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.bind(ft, gt, ht)
    plan.execute(ws)
    torch.cuda.synchronize()
    assert hdc.BatchedPlan.status(ws) == 0
    # the four phases of the launch, from the GPU's global timer
    ph = hdc.BatchedPlan.phase_ms(ws)
    assert len(ph) == 4 and all(t >= 0 for t in ph) and sum(ph) > 0
    _check(fs, gs, ht, tol)


@pytest.mark.parametrize("dt,tol", [(torch.complex128, 1e-12), (torch.complex64, 5e-5)])
def test_batched_small_rows_and_short_columns(hdc, dt, tol):
    """Many short convolutions of shared sizes, and a split convolution whose
    rows are far below a row tile and whose column axis is short (wide
    column tiles)."""
    Ls, fs, gs, ft, gt, ht = _problem(60, 40, 700, 17, dt, extra=(100,) * 9 + (97, 128, 33, 5000))
    ms = []
    for i, L in enumerate(Ls):
        M = 2 * L - 1
        ms.append(hdc.next_good_size(M) if i % 3 == 0 else hdc.next_good_size((M + 3) // 4))
    # split with rows well below a row tile: 16807 = 49 x 343 (FP64),
    # 30625 = 25 x 1225 (FP32)
    ms[-1] = 16807 if dt == torch.complex128 else 30625
    plan = hdc.BatchedPlan(Ls, ms, hdc.dtype_code(dt))
    assert plan.params[-1]["m1"] > 0 and plan.params[-1]["m2"] in (343, 1225)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.bind(ft, gt, ht)
    plan.execute(ws)
    torch.cuda.synchronize()
    assert hdc.BatchedPlan.status(ws) == 0
    _check(fs, gs, ht, tol)


def test_batched_tuned_and_graph_replay(hdc):
    dt = torch.complex128
    Ls, fs, gs, ft, gt, ht = _problem(48, 64, 8192, 11, dt)
    ms, best_ms = hdc.batched_tune(ft, gt, ht, reps=1, max_cands=3)
    assert best_ms > 0 and all(hdc.is_good_size(m) for m in ms)
    plan = hdc.BatchedPlan(Ls, ms, hdc.HDC_C128)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.bind(ft, gt, ht)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        plan.execute(ws, stream=side)          # warm (twiddles exist already)
    torch.cuda.synchronize()
    for h in ht:
        h.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        plan.execute(ws, stream=side)
    graph.replay()
    torch.cuda.synchronize()
    assert hdc.BatchedPlan.status(ws) == 0
    _check(fs, gs, ht, 1e-12)
    for h in ht:
        h.zero_()
    graph.replay()
    torch.cuda.synchronize()
    _check(fs, gs, ht, 1e-12)


def test_barrier_timeout_reports_status(hdc):
    """A barrier that waits for a block that does not exist gives up after
    its spin limit: status HDC_ERR_TIMEOUT, and the next launch is fine."""
    dt = torch.complex128
    Ls, fs, gs, ft, gt, ht = _problem(8, 64, 2048, 13, dt, extra=(9000,))
    ms = [hdc.next_good_size(2 * L - 1) for L in Ls]
    plan = hdc.BatchedPlan(Ls, ms, hdc.HDC_C128)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.bind(ft, gt, ht)
    plan.set_barrier(spin_limit=2000, extra_arrivals=1)
    plan.execute(ws)
    torch.cuda.synchronize()
    assert hdc.BatchedPlan.status(ws) == hdc.HDC_ERR_TIMEOUT
    plan.set_barrier(spin_limit=1 << 26, extra_arrivals=0)
    plan.execute(ws)
    torch.cuda.synchronize()
    assert hdc.BatchedPlan.status(ws) == 0
    _check(fs, gs, ht, 1e-12)

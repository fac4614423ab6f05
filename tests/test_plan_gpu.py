"""Plans, the parameter search, the host-buffer call and launch statistics
on the GPU, each checked against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2306_10016_gb300 import synth
from conftest import rel_max_err, check_best_timed

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


def _inputs(L, seed=0, dt=torch.complex128):
    f = synth.unit_disk(seed + 1, (L,))
    g = synth.unit_disk(seed + 2, (L,))
    return f, g, torch.from_numpy(f).cuda().to(dt), torch.from_numpy(g).cuda().to(dt)


def test_plan_modes(hdc, tmp_path):
    L = 1000
    f, g, ft, gt = _inputs(L)
    ref = oracle.conv_direct(f, g)
    for mode, kw in [(hdc.HDC_FIXED, dict(m=[256], D=[2])), (hdc.HDC_EXPLICIT, {}),
                     (hdc.HDC_TUNE_EXHAUSTIVE, dict(tuning_db=str(tmp_path / "db.txt")))]:
        pl = hdc.Plan([L], mode=mode, **kw)
        h = pl.execute(ft, gt)
        torch.cuda.synchronize()
        assert rel_max_err(h.cpu().numpy(), ref) < 1e-12, mode
    text = (tmp_path / "db.txt").read_text()
    assert " 1000 1999 |" in text
    # the second plan comes from the database: same parameters
    p1 = hdc.Plan([L], mode=hdc.HDC_TUNE_EXHAUSTIVE, tuning_db=str(tmp_path / "db.txt")).params
    p2 = hdc.Plan([L], mode=hdc.HDC_TUNE_CACHED_ONLY, tuning_db=str(tmp_path / "db.txt")).params
    assert p1 == p2


def test_tune_returns_fastest_trial(hdc):
    L = 4096
    f, g, ft, gt = _inputs(L, 10)
    best, trials = hdc.tune(ft, gt, 1, max_ratio=1.3, reps=3)
    assert trials and best[0]["ms"] > 0
    check_best_timed(best, trials)
    h = hdc.conv1d(ft, gt, best[0]["m"], D=best[0]["D"])
    torch.cuda.synchronize()
    assert rel_max_err(h.cpu().numpy(), oracle.conv_direct(f, g)) < 1e-12


def test_tune_2d_separable(hdc):
    shape = (40, 48)
    f = synth.unit_disk(31, shape)
    g = synth.unit_disk(32, shape)
    ft, gt = torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda()
    best, trials = hdc.tune(ft, gt, 2, max_ratio=1.3, reps=2)
    assert len(best) == 2
    h = hdc.conv2d(ft, gt, [b["m"] for b in best], D=[b["D"] for b in best])
    torch.cuda.synchronize()
    assert rel_max_err(h.cpu().numpy(), oracle.conv_direct(f, g)) < 1e-12


@pytest.mark.parametrize("dt,tol", [(torch.complex128, 1e-12), (torch.complex64, 5e-5)])
def test_host_buffer_call(hdc, dt, tol):
    L = 3000
    f = synth.unit_disk(41, (2, L))
    g = synth.unit_disk(42, (2, L))
    fh = torch.from_numpy(f).to(dt).pin_memory()
    gh = torch.from_numpy(g).to(dt).pin_memory()
    hh = torch.empty_like(fh).pin_memory()
    hdc.convnd_host(fh, gh, hh, 1, 1024, D=1)
    for b in range(2):
        assert rel_max_err(hh[b].numpy(), oracle.conv_direct(f[b], g[b])) < tol


def test_launch_stats(hdc):
    L = 5000
    f, g, ft, gt = _inputs(L, 20)
    hdc.conv1d(ft, gt, 1250, D=2)           # warm: twiddle tables
    torch.cuda.synchronize()
    hdc.stats_reset()
    hdc.stats_timing(True)
    n0 = hdc.total_launches()
    hdc.conv1d(ft, gt, 1250, D=2)            # q = 8 residues in 4 passes
    torch.cuda.synchronize()
    hdc.stats_timing(False)
    st = hdc.stats()
    per_kernel = sum(v["launches"] for v in st.values())
    assert hdc.total_launches() - n0 == per_kernel
    # every pass runs the residue kernel once and ends with one unfold, on its
    # own or fused with the inverse column transforms
    unf = st["k_unfold"]["launches"] + st["k_ifft_unfold_cols"]["launches"]
    assert st["k_residue_rows"]["launches"] == 4 and unf == 4
    fold = st["k_fold_fft_cols"]["launches"] + st["k_fold_fft_cols_tma"]["launches"]
    assert fold in (0, 4) and st["k_ifft_cols"]["launches"] in (0, 4)
    for k, v in st.items():
        if v["launches"]:
            assert v["ms"] > 0 and v["flops"] > 0 and v["bytes"] > 0, k


def test_fma_probe(hdc):
    assert hdc.probe_fma_peak(hdc.HDC_C128, iters=1 << 12, reps=2) > 0.1
    assert hdc.probe_fma_peak(hdc.HDC_C64, iters=1 << 12, reps=2) > 1.0


def test_cheap_tuners_random_and_proxy(hdc):
    """Random search and the height-32 rectangle return valid tuples whose
    convolution matches the oracle; random search times fewer
    configurations than the grid search; plan modes cache their choice."""
    import numpy as np
    import oracle
    from paper_2306_10016_gb300 import synth
    from conftest import rel_max_err
    shape = (96, 200)
    f = torch.from_numpy(synth.unit_disk(3101, shape)).cuda()
    g = torch.from_numpy(synth.unit_disk(3102, shape)).cuda()
    full, ftr = hdc.tune(f, g, 2, max_ratio=1.5, reps=2)
    rb, rtr = hdc.tune_random(f, g, 2, max_ratio=1.5, reps=2)
    assert 0 < len(rtr) < len(ftr)
    xb, xn = hdc.tune_proxy(f, g, 2, 32, max_ratio=1.5, reps=2)
    assert xn > 0
    ref = oracle.conv_fft(f.cpu().numpy(), g.cpu().numpy())
    for b in (rb, xb):
        h = hdc.convnd(f, g, 2, [t["m"] for t in b], D=[t["D"] for t in b]).cpu().numpy()
        assert rel_max_err(h, ref) < 1e-12
    again = hdc.tune_random(f, g, 2, max_ratio=1.5, reps=2)[0]
    assert [t["m"] for t in again] and len(again) == 2


def test_plan_modes_random_and_proxy(hdc, tmp_path):
    from paper_2306_10016_gb300 import synth
    import oracle
    from conftest import rel_max_err
    shape = [64, 150]
    f = torch.from_numpy(synth.unit_disk(3201, shape)).cuda()
    g = torch.from_numpy(synth.unit_disk(3202, shape)).cuda()
    ref = oracle.conv_fft(f.cpu().numpy(), g.cpu().numpy())
    db = str(tmp_path / "db.txt")
    for mode in (hdc.HDC_TUNE_RANDOM, hdc.HDC_TUNE_PROXY):
        pl = hdc.Plan(shape, mode=mode, tuning_db=db)
        h = pl.execute(f, g).cpu().numpy()
        assert rel_max_err(h, ref) < 1e-12
        again = hdc.Plan(shape, mode=mode, tuning_db=db)
        assert again.params == pl.params
    lines = open(db).read().splitlines()
    assert sum(" random |" in x for x in lines) == 1 and sum(" proxy |" in x for x in lines) == 1


def test_cheap_tuners_respect_the_outer_axis_limit(hdc):
    """Outer-axis candidates above hdc_max_outer_fft_size are never drawn
    (a random start there used to fail every timing of the inner axis)."""
    from paper_2306_10016_gb300 import synth
    lim = hdc.max_outer_fft_size(hdc.HDC_C128)
    f = torch.from_numpy(synth.unit_disk(3301, (2048, 40))).cuda()
    g = torch.from_numpy(synth.unit_disk(3302, (2048, 40))).cuda()
    for seed in (1, 2, 3, 4):
        best, trials = hdc.tune_random(f, g, 2, seed=seed, max_ratio=1.5, reps=1)
        assert best[0]["m"] <= lim and all(t[0]["m"] <= lim for t in trials)
    best, _ = hdc.tune(f, g, 2, max_ratio=1.5, reps=1)
    assert best[0]["m"] <= lim

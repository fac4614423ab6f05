"""Throughput of hybrid dealiased convolution on GB300.

Workload (one step): the 1-D complex FP64 sweep L in {2^10 .. 2^22} and
{3 * 2^9 .. 3 * 2^20} (25 sizes), M = 2L - 1, inputs uniform in the unit
disk (seeded), each size convolved once with its tuned hybrid parameters
(grid search of Section 4.2 run before the timed region).  The metric is
conv outputs per second over the whole sweep; the explicit-padding path
(m = nextgood(M), p = q = 1) and the FP32 path are timed the same way and
reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Under torchrun (N > 1) the job is N copies of the
sweep with distinct inputs and a batch of N x 4096 convolutions, dealt out
to the ranks by sharding.shard_batch (longest first onto the least loaded
rank; the convolutions are independent, so no data is exchanged: weak
scaling); the time is the max over ranks and value counts every rank's
outputs.  The other workloads run as replicas.

The CPU leg (rank 0, after every timed region) runs the oracle twice over:
timed on the host cores as the CPU baseline, and untimed as the FP64
reference of every result the GPU arm produced (``max_rel_err`` and the
per-size errors), which is the only use of the oracle here.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "conv outputs/s & %roofline, tuned hybrid vs explicit, FP64 err≤1e-12"
UNIT = "outputs/s"
SM_COUNT = 152
# streams the timed sweep steps issue their independent sizes over
SWEEP_STREAMS = 3
SM_MAX_MHZ = 2070.0


def _measured_hbm_gbs() -> float:
    """HBM copy bandwidth measured on this machine's GPUs (MEASURED_PEAKS.json
    beside this file), else the 6.8 TB/s fallback of an earlier measurement."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


HBM_GBS = _measured_hbm_gbs()
# FP64 / FP32 vector FMA units per SM of GB300 (2 DFMA and 128 FFMA per clock),
# 2 flops per FMA: peak = SMs x units x 2 x max SM clock.
FP64_FMA_PER_CLK = 2
FP32_FMA_PER_CLK = 128
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) over algorithmic
# bytes of one launch of the dominant kernel, from one ncu capture of its
# largest launch in the sweep (L = 2^22: k_residue_rows over 4096 rows of
# 2048 points; profiles/launches_fp64_sweep.md); the roofline's traffic per
# launch is this ratio times the step's average algorithmic bytes per launch.
# To be re-taken whenever that kernel changes (and None until then).
NCU_DRAM_PER_ALG_BYTE: dict = {"k_residue_rows": (268573184 + 90074368) / 402653184}


def _good(n: int) -> bool:
    for f in (2, 3, 5, 7):
        while n % f == 0:
            n //= f
    return n == 1


def model_flops(L: int, m: int, q: int) -> float:
    """F1 = q (15 m log2 m + 6 m + 24 L) + 2 L: three transforms, the product,
    the folds and the unfold of every residue, and the scaling."""
    return q * (15 * m * math.log2(m) + 6 * m + 24 * L) + 2 * L


def smooth_upto(n: int) -> list:
    """The 7-smooth numbers 2^a 3^b 5^c 7^d <= n."""
    out = []
    p7 = 1
    while p7 <= n:
        p5 = p7
        while p5 <= n:
            p3 = p5
            while p3 <= n:
                x = p3
                while x <= n:
                    out.append(x)
                    x *= 2
                p3 *= 3
            p5 *= 5
        p7 *= 7
    return sorted(out)


def floor_flops(L: int) -> float:
    """The least model flops over the valid tuples of one 1-D axis (M = 2L - 1):
    every 7-smooth m from 16 up to the explicit size, q = ceil(M / m)."""
    M = 2 * L - 1
    top = M
    while not _good(top):
        top += 1
    return min(model_flops(L, m, -(-M // m)) for m in smooth_upto(top) if m >= 16)


def valid_tuple_count(L: int) -> int:
    """Valid (m, p, q, D) of one axis with M = 2L - 1: every 7-smooth m from
    16 up to the explicit size, p and q derived, D in {1, 2, 4, ...} below q
    and D = q."""
    M = 2 * L - 1
    top = M
    while not _good(top):
        top += 1
    n = 0
    for m in smooth_upto(top):
        if m < 16:
            continue
        q = -(-M // m)
        n += len({d for d in (1 << k for k in range(0, 40)) if d < q} | {q})
    return n


def sweep_sizes():
    s = [1 << k for k in range(10, 23)] + [3 << k for k in range(9, 21)]
    return sorted(s)


def workload_name(dtype):
    return (f"1-D complex {dtype} sweep L=2^10..2^22 and 3*2^9..3*2^20 (25 sizes), M=2L-1, "
            "unit-disk inputs, tuned hybrid (m,p,q,D) per size")


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ oracle (CPU)

def cpu_baseline(sizes, budget_s=20.0, seed_base=0):
    """The oracle's explicitly padded FFT convolution (O2) on the host cores,
    over the sweep's sizes in increasing order until the time budget is used."""
    import oracle
    from paper_2306_10016_gb300 import synth
    oracle.lib()
    done, outs, t_tot = [], 0, 0.0
    for i, L in enumerate(sizes):
        f = synth.unit_disk(seed_base + 1 + i, (L,))
        g = synth.unit_disk(seed_base + 1001 + i, (L,))
        t0 = time.perf_counter()
        oracle.conv_fft(f, g)
        dt = time.perf_counter() - t0
        t_tot += dt
        outs += L
        done.append(L)
        if t_tot > budget_s:
            break
    return {"value": outs / t_tot, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"explicit zero-padded radix-2 FFT convolution (FP64, OpenMP) of the sweep sizes "
                      f"{done[0]}..{done[-1]} ({len(done)} of {len(sizes)} sizes, each once), {t_tot:.1f} s"}


def rel_max_err(x, ref) -> float:
    """max |x - ref| / max |ref| (the per-result error of Section 2.3's
    convolution, Eq. 4, against its FP64 reference)."""
    import numpy as np
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = float(np.max(np.abs(ref))) if ref.size else 0.0
    num = float(np.max(np.abs(x - ref))) if ref.size else 0.0
    return num / den if den > 0 else num


def oracle_errors(pending):
    """The CPU leg's second part, after every timed region: the FP64 oracle's
    reference of each result the GPU arm produced, and the result's relative
    max-norm error against it.  pending: (name, result, key, ref_fn) with
    ref_fn(oracle) -> reference; references are cached by key, so the FP64,
    explicit, FP32 and end-to-end results of one input share one.  A key
    starting with "int:" marks integer-valued inputs, whose FP64 result must
    round to the exact integer convolution: those report exact = True/False."""
    import numpy as np
    import oracle
    oracle.lib()
    cache, out = {}, {}
    t0 = time.perf_counter()
    for name, got, key, ref_fn in pending:
        if key not in cache:
            cache[key] = ref_fn(oracle)
        ref = cache[key]
        if isinstance(ref, list):
            out[name] = max(rel_max_err(a, b) for a, b in zip(got, ref))
        elif key.startswith("int:"):
            hre, him = ref
            out[name] = {"exact": bool(np.array_equal(np.rint(got.real).astype(np.int64), hre)
                                       and np.array_equal(np.rint(got.imag).astype(np.int64), him)),
                         "max_abs_err": float(np.max(np.abs(got - (hre + 1j * him))))}
        else:
            out[name] = rel_max_err(got, ref)
    return out, time.perf_counter() - t0


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2306_10016_gb300 import synth
    oracle.lib()
    sizes = [L for L in sweep_sizes() if L <= (1 << 16)]
    inputs = [(synth.unit_disk(1 + i, (L,)), synth.unit_disk(1001 + i, (L,))) for i, L in enumerate(sizes)]
    for _ in range(max(0, args.warmup)):
        for f, g in inputs[:3]:
            oracle.conv_fft(f, g)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for f, g in inputs:
            oracle.conv_fft(f, g)
        ts.append(time.perf_counter() - t0)
    outs = sum(sizes)
    value = outs / (sum(ts) / len(ts))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name("FP64"), "reference_sample": f"sizes {sizes[0]}..{sizes[-1]} "
                   f"({len(sizes)} of 25) per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"explicit zero-padded radix-2 FFT convolution (FP64) of the sweep sizes "
                                   f"{sizes[0]}..{sizes[-1]} per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hdc", choices=["hdc", "reference"])
    ap.add_argument("--tuning-db", default=os.environ.get(
        "HDC_TUNING_DB", os.path.join(os.path.expanduser("~"), ".cache", "hdc", "tuning.txt")))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sizes", default="", help="comma-separated L list (default: the full sweep)")
    ap.add_argument("--eager", action="store_true",
                    help="launch every timed step directly instead of replaying a captured CUDA graph "
                         "(same work; for profilers that do not follow graph replays)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_2306_10016_gb300 as hdc
    from paper_2306_10016_gb300 import sharding, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    hdc.build()
    hdc.lib()

    base_sizes = [int(x) for x in args.sizes.split(",")] if args.sizes else sweep_sizes()
    # N copies of the sweep, dealt out by model cost; a unit is (copy, size
    # index) and its inputs are seeded by both, so rank 0 of a 1-rank run
    # sees the single copy 0
    mine = sharding.shard_copies([sharding.model_flops(L, L, 2) for L in base_sizes], world)[rank]
    sizes = [base_sizes[i] for _, i in mine]
    total_outs = world * sum(base_sizes)
    os.makedirs(os.path.dirname(args.tuning_db), exist_ok=True)
    # results to check against the oracle once every timed region is over:
    # (name, result on the host, reference key, reference builder)
    pending = []

    def sweep_inputs(i, L):
        c, ib = mine[i]
        off = ib + 100003 * c
        return synth.unit_disk(synth.BASE_SEED + 10 + off, (L,)), synth.unit_disk(synth.BASE_SEED + 1010 + off, (L,))

    def sweep_ref(i, L):
        return lambda o: o.conv_fft(*sweep_inputs(i, L))

    def check_sweep(tag, ins):
        for i, (L, (_, _, h)) in enumerate(zip(sizes, ins)):
            pending.append((f"{tag}/L={L}", h.cpu().numpy().astype(np.complex128), f"sweep{i}", sweep_ref(i, L)))

    def make_inputs(tdt):
        ins = []
        for i, L in enumerate(sizes):
            fn, gn = sweep_inputs(i, L)
            f = torch.from_numpy(fn).to(dev, tdt)
            g = torch.from_numpy(gn).to(dev, tdt)
            ins.append((f, g, torch.empty_like(f)))
        return ins

    def make_plans(dtype, mode):
        plans = []
        for L in sizes:
            db = args.tuning_db if mode == hdc.HDC_TUNE_EXHAUSTIVE else None
            plans.append(hdc.Plan([L], dtype=dtype, mode=mode, tuning_db=db))
        return plans

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    def time_sweep(plans, ins, steps, warmup, stats=False, nvtx=None, reps=1, nstreams=1):
        """Warm up eagerly, capture one step (every size once, `reps` times) in
        a CUDA graph, then time `steps` replays with events, flushing L2 before
        each; returns the time per repetition.  nstreams > 1: the sizes of a
        step are independent convolutions, issued over that many streams
        (forked from the step's stream and joined back, a workspace each) in
        the order small-large-small, so the short launches of the small sizes
        run beside the others instead of one after another."""
        nst = 1 if (stats or len(plans) == 1) else nstreams
        wsb = max(p.workspace_bytes for p in plans)
        wss = [torch.empty(wsb, dtype=torch.uint8, device=dev) for _ in range(nst)]
        ws = wss[0]
        side = torch.cuda.Stream(dev)
        extra = [torch.cuda.Stream(dev) for _ in range(nst - 1)]
        by_size = sorted(range(len(plans)), key=lambda i: ins[i][0].numel())
        order = by_size[0::2] + by_size[1::2][::-1]

        def step(st):
            if nst == 1:
                for p, (f, g, h) in zip(plans, ins):
                    p.execute(f, g, out=h, workspace=ws, stream=st)
                return
            for s_ in extra:
                s_.wait_stream(st)
            streams = [st] + extra
            for k_, i in enumerate(order):
                f, g, h = ins[i]
                plans[i].execute(f, g, out=h, workspace=wss[k_ % nst], stream=streams[k_ % nst])
            for s_ in extra:
                st.wait_stream(s_)

        with torch.cuda.stream(side):
            for _ in range(warmup):
                step(side)
        torch.cuda.synchronize(dev)
        if stats:
            # one eager step with timing fills the library's event pool, so the
            # capture below creates no events
            hdc.stats_timing(True)
            with torch.cuda.stream(side):
                step(side)
            torch.cuda.synchronize(dev)
            hdc.stats_reset()
        n0 = hdc.total_launches()
        st = torch.cuda.current_stream(dev)
        if args.eager:
            graph = None

            def replay():
                for _ in range(reps):
                    step(st)
        else:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                for _ in range(reps):
                    step(side)
            replay = graph.replay
        per_step = hdc.total_launches() - n0
        if stats and not args.eager:
            hdc.stats_timing(False)
        replay()
        torch.cuda.synchronize(dev)
        if stats and args.eager:
            hdc.stats_reset()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        if nvtx:
            torch.cuda.nvtx.range_push(nvtx)
        n1 = hdc.total_launches()
        ev = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            replay()
            e1.record(st)
            ev.append((e0, e1))
        torch.cuda.synchronize(dev)
        if args.eager:
            per_step = (hdc.total_launches() - n1) // steps
        if stats and args.eager:
            hdc.stats_timing(False)
        if nvtx:
            torch.cuda.nvtx.range_pop()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)
        ms = [a.elapsed_time(b) / reps for a, b in ev]
        kst = None
        if stats:
            try:
                kst = hdc.stats()     # event pairs of the last replay (graph) or of every step (eager)
            except Exception:
                kst = None
            if kst is not None and args.eager:
                for v in kst.values():   # per step, as after a replay
                    v["ms"] /= steps
                    v["flops"] /= steps
                    v["launches"] //= steps
        del graph
        return sum(ms) / len(ms), per_step * steps, ms, kst

    # --- measured FMA peaks (context beside the unit-count peak)
    fp64_probe = hdc.probe_fma_peak(hdc.HDC_C128, iters=1 << 14, device=dev)

    # --- FP64 tuned hybrid (headline)
    t_tune0 = time.perf_counter()
    ins64 = make_inputs(torch.complex128)
    plans64 = make_plans(hdc.HDC_C128, hdc.HDC_TUNE_EXHAUSTIVE)
    tune_s = time.perf_counter() - t_tune0
    sampler = ClockSampler(local)
    sampler.start()
    # the headline and the explicit comparison are timed without per-kernel
    # events (event records in the graph would add to every launch); the
    # per-kernel split of the roofline comes from a second, instrumented run
    ms64, launches, ms_list, _ = time_sweep(plans64, ins64, args.steps, args.warmup, nvtx="hdc_fp64_timed",
                                            nstreams=SWEEP_STREAMS)
    clocks = sampler.stop()
    check_sweep("sweep_fp64", ins64)
    _, _, _, kstats = time_sweep(plans64, ins64, args.steps, 1, stats=True)
    if kstats is None:
        raise RuntimeError("per-kernel event times unavailable")

    # max over ranks
    def rank_max(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms64 = rank_max(ms64)
    outs = sum(sizes)
    value = total_outs / (ms64 * 1e-3)

    # --- explicit padding, FP64
    plans_ex = make_plans(hdc.HDC_C128, hdc.HDC_EXPLICIT)
    ms_ex, _, _, _ = time_sweep(plans_ex, ins64, args.steps, args.warmup, nstreams=SWEEP_STREAMS)
    ms_ex = rank_max(ms_ex)
    check_sweep("explicit_fp64", ins64)

    # integer inputs in [-8, 8] through the tuned plans of four sweep sizes
    # (one untimed call each): the FP64 result must round to the exact
    # integer convolution
    for L in [x for x in (1 << 16, 1 << 20, 3 << 20, 1 << 22) if x in sizes]:
        i = sizes.index(L)
        fr, fi = synth.small_ints(synth.BASE_SEED + 20 + i, (L,))
        gr, gi = synth.small_ints(synth.BASE_SEED + 1020 + i, (L,))
        fz = torch.from_numpy(synth.ints_to_complex(fr, fi)).to(dev)
        gz = torch.from_numpy(synth.ints_to_complex(gr, gi)).to(dev)
        hz = torch.empty_like(fz)
        wz = torch.empty(plans64[i].workspace_bytes, dtype=torch.uint8, device=dev)
        plans64[i].execute(fz, gz, out=hz, workspace=wz)
        torch.cuda.synchronize(dev)
        pending.append((f"integer_fp64/L={L}", hz.cpu().numpy(), f"int:{L}",
                        lambda o, a=(fr, fi, gr, gi): o.conv_int_exact(*a, method="ntt")))
        del fz, gz, hz, wz

    # --- per-size hybrid vs explicit (device time, FP64)
    def ab_times(pa, pb, f, g, h, n=45):
        """The calls of two plans on the same data, each captured in a CUDA
        graph with ONE shared workspace (so both run on the same addresses),
        then replayed alternately (A B, B A, ...), each replay after an L2
        flush, n times each; the times of each."""
        ws = torch.empty(max(1, pa.workspace_bytes, pb.workspace_bytes), dtype=torch.uint8, device=dev)
        side = torch.cuda.Stream(dev)
        graphs = []
        for p_ in (pa, pb):
            with torch.cuda.stream(side):
                p_.execute(f, g, out=h, workspace=ws, stream=side)
            torch.cuda.synchronize(dev)
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=side):
                p_.execute(f, g, out=h, workspace=ws, stream=side)
            gr.replay()
            graphs.append(gr)
        torch.cuda.synchronize(dev)
        st = torch.cuda.current_stream(dev)
        ev = ([], [])
        for i in range(n):
            # A B, then B A: the order within a pair alternates
            for k in ((0, 1) if i % 2 == 0 else (1, 0)):
                gr = graphs[k]
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                gr.replay()
                e1.record(st)
                ev[k].append((e0, e1))
        torch.cuda.synchronize(dev)
        del graphs
        return [[a.elapsed_time(b) for a, b in e] for e in ev]

    # per size, the tuned and the explicit tuple on the same workspace,
    # replayed alternately (45 each, L2 flushed before each; median).  Where
    # the tuner chose the explicit tuple itself, the two plans run the same
    # launches, and both report the median of all 90 times
    per_size = []
    for L, pt, pe, (f, g, h) in zip(sizes, plans64, plans_ex, ins64):
        th, te = ab_times(pt, pe, f, g, h)
        prm = pt.params[0]
        same = prm["q"] == 1 and prm["m"] == pe.params[0]["m"]
        th_ms, te_ms = (statistics.median(th + te),) * 2 if same else (statistics.median(th), statistics.median(te))
        per_size.append({"L": L, "m": prm["m"], "p": prm["p"], "q": prm["q"], "D": prm["D"],
                         "hybrid_ms": round(th_ms, 5),
                         "explicit_ms": round(te_ms, 5),
                         "same_tuple_as_explicit": same,
                         "valid_tuples": valid_tuple_count(L), "timed_tuples": pt.timed})
    del ins64

    # --- FP32 tuned hybrid
    ins32 = make_inputs(torch.complex64)
    plans32 = make_plans(hdc.HDC_C64, hdc.HDC_TUNE_EXHAUSTIVE)
    ms32, _, _, _ = time_sweep(plans32, ins32, args.steps, args.warmup, nstreams=SWEEP_STREAMS)
    ms32 = rank_max(ms32)
    check_sweep("sweep_fp32", ins32)
    _, _, _, kstats32 = time_sweep(plans32, ins32, 1, 1, stats=True)
    # per size, the tuned FP32 call alone (15 single-call replays after an L2
    # flush each, median), with the route's launches
    per_size32 = []
    for L, pt, (f, g, h) in zip(sizes, plans32, ins32):
        hdc.stats_reset()
        _, nl, tl, _ = time_sweep([pt], [(f, g, h)], 15, 1, reps=1)
        prm = pt.params[0]
        per_size32.append({"L": L, "m": prm["m"], "p": prm["p"], "q": prm["q"], "D": prm["D"],
                           "ms": round(statistics.median(tl), 5), "launches": nl // 15})
    del ins32

    # --- batched: 4096 convolutions, L log-uniform in [64, 65536], one
    # persistent launch per step, replayed from a CUDA graph
    def batched_run(tdt, dcode, nconv_rank=4096):
        # the job's batch is N x 4096 lengths, dealt out by model cost; this
        # rank's inputs are seeded by the rank
        Lg = [int(x) for x in synth.log_uniform_lengths(synth.BASE_SEED + 4, nconv_rank * world, 64, 65536)]
        Ls = [Lg[i] for i in sharding.shard_batch([sharding.model_flops(L, L, 2) for L in Lg], world)[rank]]
        nconv = len(Ls)
        tot = sum(Ls)
        tot_job = sum(Lg)
        seed_in = synth.BASE_SEED + 40 + 7919 * rank
        fa = torch.from_numpy(synth.unit_disk(seed_in, (tot,))).to(dev, tdt)
        ga = torch.from_numpy(synth.unit_disk(seed_in + 1, (tot,))).to(dev, tdt)
        ha = torch.empty_like(fa)
        offs = np.concatenate([[0], np.cumsum(Ls)])
        fs = [fa[offs[i]:offs[i + 1]] for i in range(nconv)]
        gs = [ga[offs[i]:offs[i + 1]] for i in range(nconv)]
        hs = [ha[offs[i]:offs[i + 1]] for i in range(nconv)]
        # the convolutions checked against the oracle: every one with
        # L <= 2048 and a seeded sample of 64 longer ones
        rng = np.random.default_rng(synth.BASE_SEED + 4)
        longer = [i for i in range(nconv) if Ls[i] > 2048]
        sel = [i for i in range(nconv) if Ls[i] <= 2048] + sorted(
            rng.choice(longer, size=min(64, len(longer)), replace=False).tolist())

        def batched_ref(o):
            fa_n = synth.unit_disk(seed_in, (tot,))
            ga_n = synth.unit_disk(seed_in + 1, (tot,))
            return [o.conv_fft(fa_n[offs[i]:offs[i + 1]], ga_n[offs[i]:offs[i + 1]]) for i in sel]

        t0 = time.perf_counter()
        ms_t, _ = hdc.batched_tune(fs, gs, hs, reps=3, max_cands=15)
        tune_b = time.perf_counter() - t0
        res = {}
        for name, mlist in (("tuned", ms_t), ("explicit", [hdc.next_good_size(2 * L - 1) for L in Ls])):
            plan = hdc.BatchedPlan(Ls, mlist, dcode)
            wsb = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
            plan.bind(fs, gs, hs)
            side = torch.cuda.Stream(dev)
            with torch.cuda.stream(side):
                for _ in range(max(1, args.warmup)):
                    plan.execute(wsb, stream=side)
            torch.cuda.synchronize(dev)
            st = torch.cuda.current_stream(dev)
            if args.eager:
                graph = None
                replay = lambda: plan.execute(wsb, stream=st)   # noqa: E731
            else:
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=side):
                    plan.execute(wsb, stream=side)
                replay = graph.replay
            ev = []
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                replay()
                e1.record(st)
                ev.append((e0, e1))
            torch.cuda.synchronize(dev)
            ok = hdc.BatchedPlan.status(wsb) == 0
            phases = [round(x, 4) for x in hdc.BatchedPlan.phase_ms(wsb)]
            hh = ha.cpu().numpy().astype(np.complex128)
            pending.append((f"batched_{'fp64' if dcode == hdc.HDC_C128 else 'fp32'}_{name}",
                            [hh[offs[i]:offs[i + 1]] for i in sel], "batched", batched_ref))
            del hh
            msb = rank_max(sum(a.elapsed_time(b) for a, b in ev) / len(ev))
            fl = sum(pp["q"] * (15 * pp["m"] * math.log2(pp["m"]) + 6 * pp["m"] + 24 * pp["L"]) + 2 * pp["L"]
                     for pp in plan.params)
            res[name] = {"value": tot_job / (msb * 1e-3), "ms": round(msb, 4), "status_ok": ok,
                         "phase_ms_last_replay": phases,
                         "model_tflops": round(fl / (msb * 1e-3) / 1e12, 4)}
            del graph, plan, wsb
        res["convolutions"] = nconv
        res["checked_against_oracle"] = len(sel)
        res["outputs"] = tot
        res["lengths"] = Ls
        res["tuning_s"] = round(tune_b, 1)
        return res

    batched64 = batched_run(torch.complex128, hdc.HDC_C128)
    blens = batched64.pop("lengths")
    batched64["roofline_frac"] = round(batched64["tuned"]["model_tflops"] / (
        SM_COUNT * FP64_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12), 4)
    batched32 = batched_run(torch.complex64, hdc.HDC_C64)
    batched32.pop("lengths")
    batched32["roofline_frac"] = round(batched32["tuned"]["model_tflops"] / (
        SM_COUNT * FP32_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12), 4)

    # --- the single small convolution: L = 1024, M = 2047, fixed (m, p, q, D)
    # = (512, 2, 4, 1) (p = 2, the least p with p m >= L); latency of one call,
    # and throughput of 16384 copies as the rows of one call
    def config1():
        L1 = 1024
        f1 = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 1, (16384, L1))).to(dev)
        g1 = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 101, (16384, L1))).to(dev)
        h1 = torch.empty_like(f1)
        ws1 = torch.empty(hdc.workspace_size([L1], [2 * L1 - 1], [512], p=[2], q=[4], D=[1], batch=16384),
                          dtype=torch.uint8, device=dev)
        st = torch.cuda.current_stream(dev)
        one = lambda: hdc.convnd(f1[0], g1[0], 1, [512], p=[2], q=[4], D=[1], out=h1[0], workspace=ws1,  # noqa: E731
                                 stream=st)
        for _ in range(5):
            one()
        torch.cuda.synchronize(dev)
        # eager: the Python call, its argument checks and eight launches
        # (four passes of rows + unfold) as the stream sees them
        lat = []
        for _ in range(21):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            one()
            e1.record(st)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1) * 1e3)
        lat.sort()
        # the same call captured once in a CUDA graph and replayed: the
        # device-side latency
        ms_one, _ = graph_time(lambda s_: hdc.convnd(f1[0], g1[0], 1, [512], p=[2], q=[4], D=[1], out=h1[0],
                                                     workspace=ws1, stream=s_), 21)
        msr, _ = graph_time(lambda s_: hdc.convnd(f1, g1, 1, [512], p=[2], q=[4], D=[1], out=h1, workspace=ws1,
                                                  stream=s_), max(args.steps, 5))
        rows = [0, 1, 8191, 16383]
        hrows = h1[rows].cpu().numpy()

        def c1_ref(o):
            fn = synth.unit_disk(synth.BASE_SEED + 1, (16384, L1))
            gn = synth.unit_disk(synth.BASE_SEED + 101, (16384, L1))
            return [o.conv_direct(fn[r], gn[r]) for r in rows]

        pending.append(("config1_fp64", [hrows[k] for k in range(len(rows))], "config1", c1_ref))
        return {"params": {"m": 512, "p": 2, "q": 4, "D": 1},
                "latency_us": {"graph_replay": round(ms_one * 1e3, 2),
                               "eager_call_median": round(lat[10], 2), "eager_call_p10": round(lat[2], 2),
                               "eager_call_p90": round(lat[18], 2), "calls": 21},
                "replicated": {"copies": 16384, "ms": round(msr, 4),
                               "value": world * 16384 * L1 / (msr * 1e-3)}}

    # --- the sweep against the roofline of its least-flop tuples: T* = max(
    # 3 sum L * bytes / HBM, sum F_floor / vector peak), both dtypes (the
    # tuned and the explicit paths are scored against the same T*)
    def floor_roofline(ms, es, peak_flops, Ls=None):
        Ls = sizes if Ls is None else Ls
        ff = sum(floor_flops(L) for L in Ls)
        bb = 3.0 * sum(Ls) * es
        t_star = max(bb / (HBM_GBS * 1e9), ff / peak_flops)
        return {"frac": round(t_star / (ms * 1e-3), 4), "t_star_ms": round(t_star * 1e3, 4),
                "floor_gflop": round(ff / 1e9, 3), "bytes_mb": round(bb / 1e6, 1),
                "basis": "T* = max(3 sum L x element bytes / measured HBM, sum of least model flops over valid "
                         "tuples / vector FMA peak), over the measured step time"}

    # --- N-D and Hermitian configurations (FP64): tuned 2-D 1024^2 and 3-D
    # 128^3, and the centered Hermitian 2-D convolution of 1024^2 real fields
    # (K = 512 modes per axis, padding 3/2); each timed as graph replays
    peak64 = SM_COUNT * FP64_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12

    def graph_time(run, steps):
        side = torch.cuda.Stream(dev)
        with torch.cuda.stream(side):
            for _ in range(max(1, args.warmup)):
                run(side)
        torch.cuda.synchronize(dev)
        hdc.stats_reset()
        st = torch.cuda.current_stream(dev)
        if args.eager:
            graph = None
            run(st)
            replay = lambda: run(st)   # noqa: E731
        else:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                run(side)
            replay = graph.replay
        fl = sum(v["flops"] for v in hdc.stats().values())
        ev = []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            replay()
            e1.record(st)
            ev.append((e0, e1))
        torch.cuda.synchronize(dev)
        del graph
        # the replicated workloads: the slowest rank's time
        return rank_max(sum(a.elapsed_time(b) for a, b in ev) / len(ev)), fl

    nd = {}
    for name, shape in (("2d_1024x1024", (1024, 1024)), ("3d_128x128x128", (128, 128, 128))):
        f = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 30, shape)).to(dev)
        g = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 31, shape)).to(dev)
        h = torch.empty_like(f)
        t0 = time.perf_counter()
        best, _ = hdc.tune(f, g, len(shape), max_ratio=1.3, reps=5)
        tt = time.perf_counter() - t0
        mv = [b["m"] for b in best]
        Dv = [b["D"] for b in best]
        nbytes = hdc.workspace_size(list(shape), [2 * x - 1 for x in shape], mv, D=Dv)
        wsn = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        msn, fl = graph_time(lambda s_: hdc.convnd(f, g, len(shape), mv, D=Dv, out=h, workspace=wsn, stream=s_),
                             args.steps)
        outs_n = int(np.prod(shape))
        pending.append((f"nd_fp64/{name}", h.cpu().numpy(), f"nd:{name}",
                        lambda o, sh=shape: o.conv_fft(synth.unit_disk(synth.BASE_SEED + 30, sh),
                                                       synth.unit_disk(synth.BASE_SEED + 31, sh))))
        nd[name] = {"value": world * outs_n / (msn * 1e-3), "ms": round(msn, 4), "m": mv, "D": Dv,
                    "model_tflops": round(fl / (msn * 1e-3) / 1e12, 4),
                    "roofline_frac": round(fl / (msn * 1e-3) / 1e12 / peak64, 4), "tuning_s": round(tt, 1)}
        del f, g, h, wsn
    K = 512
    fh = torch.from_numpy(synth.hermitian_normal(synth.BASE_SEED + 32, K)).to(dev)
    gh = torch.from_numpy(synth.hermitian_normal(synth.BASE_SEED + 33, K)).to(dev)
    hh = torch.empty_like(fh)
    herm = {}
    # m per axis from K, 3K/2, 3K (q = 3, 2, 1 for M = 3K - 2), every pair
    for mx in (K, 3 * K // 2, 3 * K):
        for my in (K, 3 * K // 2, 3 * K):
            try:
                msh, fl = graph_time(lambda s_: hdc.conv2d_hermitian(fh, gh, m=(mx, my), out=hh, stream=s_),
                                     args.steps)
            except hdc.HDCError:
                continue
            key = f"{mx}x{my}"
            herm[key] = {"ms": round(msh, 4), "model_tflops": round(fl / (msh * 1e-3) / 1e12, 4)}
            pending.append((f"hermitian_fp64/m={key}", hh.cpu().numpy(), "herm",
                            lambda o: o.conv_hermitian_fft(synth.hermitian_normal(synth.BASE_SEED + 32, K),
                                                           synth.hermitian_normal(synth.BASE_SEED + 33, K))))
    bm = min(herm, key=lambda k: herm[k]["ms"])
    nd["hermitian_2d_K512"] = {"value": world * (2 * K - 1) * K / (herm[bm]["ms"] * 1e-3), "ms": herm[bm]["ms"],
                               "m": [int(v) for v in bm.split("x")], "model_tflops": herm[bm]["model_tflops"],
                               "roofline_frac": round(herm[bm]["model_tflops"] / peak64, 4),
                               "outputs": (2 * K - 1) * K, "by_m": herm}
    del fh, gh, hh
    cfg1 = config1()
    batched64["floor"] = floor_roofline(batched64["tuned"]["ms"], 16, peak64 * 1e12, blens)
    batched32["floor"] = floor_roofline(batched32["tuned"]["ms"], 8,
                                        SM_COUNT * FP32_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6, blens)

    # --- unequal lengths (Section 3.5, FP64): g of 2^22 points with f of
    # 2^10, 2^16 and 2^20 points, first 2^22 outputs.  Residue matching tuned
    # over (m, lam, D); beside it the best lam = 1 tuple of the same search
    # and the equal-length path on f zero-padded to g's length (M = 2 Lg - 1,
    # tuned), the way a caller without the unequal algorithm would run it.
    uneq = {}
    Lg = 1 << 22
    gu = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 40, (Lg,))).to(dev)
    hu = torch.empty_like(gu)
    for lf_log in (10, 16, 20):
        Lf = 1 << lf_log
        fu = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 41 + lf_log, (Lf,))).to(dev)

        def uneq_ref(o, Lf=Lf, lf_log=lf_log):
            fpad = np.zeros(Lg, dtype=np.complex128)
            fpad[:Lf] = synth.unit_disk(synth.BASE_SEED + 41 + lf_log, (Lf,))
            return o.conv_fft(fpad, synth.unit_disk(synth.BASE_SEED + 40, (Lg,)))

        t0 = time.perf_counter()
        bu, tru = hdc.tune_unequal(fu, gu, 1, max_ratio=1.5, reps=2)
        ttu = time.perf_counter() - t0
        lam1 = [t[0] for t in tru if t[0]["lam"] == 1]
        rows = {"matched": bu[0]}
        if lam1:
            rows["lam1"] = min(lam1, key=lambda t: t["ms"])
        res = {}
        for key, b in rows.items():
            nbu = hdc.workspace_size_unequal([Lf], [Lg], [b["m"]], [b["lam"]], D=[b["D"]])
            wsu = torch.empty(max(1, nbu), dtype=torch.uint8, device=dev)
            msu, flu = graph_time(lambda s_: hdc.convnd_unequal(fu, gu, 1, b["m"], b["lam"], D=b["D"], out=hu,
                                                                workspace=wsu, stream=s_), args.steps)
            res[key] = {"ms": round(msu, 4), "m": b["m"], "lam": b["lam"], "q": b["q"], "D": b["D"],
                        "model_tflops": round(flu / (msu * 1e-3) / 1e12, 4)}
            pending.append((f"unequal_fp64/Lf=2^{lf_log}/{key}", hu.cpu().numpy(), f"uneq:{lf_log}", uneq_ref))
            del wsu
        fpad = torch.zeros_like(gu)
        fpad[:Lf] = fu
        bp, _ = hdc.tune(fpad, gu, 1, max_ratio=1.3, reps=2)
        nbp = hdc.workspace_size([Lg], [2 * Lg - 1], [bp[0]["m"]], D=[bp[0]["D"]])
        wsp = torch.empty(nbp, dtype=torch.uint8, device=dev)
        msp, flp = graph_time(lambda s_: hdc.convnd(fpad, gu, 1, [bp[0]["m"]], D=[bp[0]["D"]], out=hu,
                                                    workspace=wsp, stream=s_), args.steps)
        res["padded_equal"] = {"ms": round(msp, 4), "m": bp[0]["m"], "q": bp[0]["q"], "D": bp[0]["D"],
                               "model_tflops": round(flp / (msp * 1e-3) / 1e12, 4)}
        pending.append((f"unequal_fp64/Lf=2^{lf_log}/padded_equal", hu.cpu().numpy(), f"uneq:{lf_log}", uneq_ref))
        best_ms = res["matched"]["ms"]
        uneq[f"Lf2^{lf_log}_Lg2^22"] = {
            "value": world * Lg / (best_ms * 1e-3), "ms": best_ms,
            "roofline_frac": round(res["matched"]["model_tflops"] / peak64, 4),
            "speedup_vs_padded": round(res["padded_equal"]["ms"] / best_ms, 4),
            "tuning_s": round(ttu, 1), "candidates_timed": len(tru), **{k: v for k, v in res.items()}}
        del fu, fpad, wsp
    del gu, hu

    # --- multi-convolution (FP64), inputs of 2^20 points: the n-fold
    # convolution of n = 3 and 4 inputs in one residue pass (tuned) against
    # chaining n - 1 tuned two-input convolutions of the running result; the
    # sum of n/2 pairwise convolutions (n = 4, 8) in one pass against n/2
    # tuned two-input convolutions summed by torch
    multi = {}
    Lm = 1 << 20
    for op, nin in (("product", 3), ("product", 4), ("dot", 4), ("dot", 8)):
        xs = [torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 50 + i, (Lm,))).to(dev) for i in range(nin)]
        hm = torch.empty_like(xs[0])
        t0 = time.perf_counter()
        bm_, _ = hdc.tune_multi(xs, 1, op=op, max_ratio=1.3, reps=2)
        ttm = time.perf_counter() - t0
        nbm = hdc.workspace_size_multi(nin, [Lm], [bm_[0]["m"]], op=op, D=[bm_[0]["D"]])
        wsm = torch.empty(nbm, dtype=torch.uint8, device=dev)
        msm, flm = graph_time(lambda s_: hdc.convnd_multi(xs, 1, [bm_[0]["m"]], op=op, D=[bm_[0]["D"]], out=hm,
                                                          workspace=wsm, stream=s_), args.steps)

        def multi_ref(o, op=op, nin=nin):
            xn = [synth.unit_disk(synth.BASE_SEED + 50 + i, (Lm,)) for i in range(nin)]
            if op == "product":
                acc = xn[0]
                for x in xn[1:]:
                    acc = o.conv_fft(acc, x)     # first Lm outputs depend on first Lm only
                return acc
            return sum(o.conv_fft(xn[i], xn[i + 1]) for i in range(0, nin, 2))

        pending.append((f"multi_fp64/{op}_n{nin}", hm.cpu().numpy(), f"multi:{op}{nin}", multi_ref))
        bp2, _ = hdc.tune(xs[0], xs[1], 1, max_ratio=1.3, reps=2)
        nb2 = hdc.workspace_size([Lm], [2 * Lm - 1], [bp2[0]["m"]], D=[bp2[0]["D"]])
        ws2 = torch.empty(nb2, dtype=torch.uint8, device=dev)
        tmp = [torch.empty_like(xs[0]), torch.empty_like(xs[0])]

        def chain(s_):
            cur = xs[0]
            for i in range(1, nin):
                nxt = tmp[i % 2]
                hdc.convnd(cur, xs[i], 1, [bp2[0]["m"]], D=[bp2[0]["D"]], out=nxt, workspace=ws2, stream=s_)
                cur = nxt

        def separate(s_):
            hdc.convnd(xs[0], xs[1], 1, [bp2[0]["m"]], D=[bp2[0]["D"]], out=tmp[0], workspace=ws2, stream=s_)
            for i in range(2, nin, 2):
                hdc.convnd(xs[i], xs[i + 1], 1, [bp2[0]["m"]], D=[bp2[0]["D"]], out=tmp[1], workspace=ws2,
                           stream=s_)
                with torch.cuda.stream(s_):
                    tmp[0].add_(tmp[1])

        msc, flc = graph_time(chain if op == "product" else separate, args.steps)
        base = "chained_pairwise" if op == "product" else "separate_pairs_summed"
        multi[f"{op}_n{nin}_L2^20"] = {
            "value": world * Lm / (msm * 1e-3), "ms": round(msm, 4), "m": bm_[0]["m"], "q": bm_[0]["q"],
            "D": bm_[0]["D"], "model_tflops": round(flm / (msm * 1e-3) / 1e12, 4),
            "roofline_frac": round(flm / (msm * 1e-3) / 1e12 / peak64, 4), "tuning_s": round(ttm, 1),
            base: {"ms": round(msc, 4), "m": bp2[0]["m"], "q": bp2[0]["q"], "D": bp2[0]["D"]},
            "speedup": round(msc / msm, 4)}
        del xs, hm, wsm, ws2, tmp

    # --- real inputs (FP64): convolution of real sequences by the packed
    # transform of f + i g and conjugate residue pairs (tuned), against the
    # complex path on the same data held as complex arrays (tuned)
    real = {}
    for name, shape in (("1d_2^20", (1 << 20,)), ("1d_2^22", (1 << 22,)), ("2d_1024x1024", (1024, 1024))):
        dims = len(shape)
        z = synth.unit_disk(synth.BASE_SEED + 60, shape)
        fr = torch.from_numpy(np.ascontiguousarray(z.real)).to(dev)
        gr = torch.from_numpy(np.ascontiguousarray(z.imag)).to(dev)
        hr = torch.empty_like(fr)
        t0 = time.perf_counter()
        br, _ = hdc.tune_real(fr, gr, dims, max_ratio=1.3, reps=2)
        ttr = time.perf_counter() - t0
        nbr = hdc.workspace_size_real(list(shape), [b["m"] for b in br], D=[b["D"] for b in br])
        wsr = torch.empty(nbr, dtype=torch.uint8, device=dev)
        msr, flr = graph_time(lambda s_: hdc.convnd_real(fr, gr, dims, [b["m"] for b in br], D=[b["D"] for b in br],
                                                         out=hr, workspace=wsr, stream=s_), args.steps)

        def real_ref(o, sh=shape):
            zz = synth.unit_disk(synth.BASE_SEED + 60, sh)
            return o.conv_fft(zz.real.astype(np.complex128), zz.imag.astype(np.complex128)).real

        pending.append((f"real_fp64/{name}", hr.cpu().numpy(), f"real:{name}", real_ref))
        fc = fr.to(torch.complex128)
        gc = gr.to(torch.complex128)
        hc = torch.empty_like(fc)
        bc, _ = hdc.tune(fc, gc, dims, max_ratio=1.3, reps=2)
        nbc = hdc.workspace_size(list(shape), [2 * x - 1 for x in shape], [b["m"] for b in bc], D=[b["D"] for b in bc])
        wsc = torch.empty(nbc, dtype=torch.uint8, device=dev)
        msc, _ = graph_time(lambda s_: hdc.convnd(fc, gc, dims, [b["m"] for b in bc], D=[b["D"] for b in bc], out=hc,
                                                  workspace=wsc, stream=s_), args.steps)
        pending.append((f"real_fp64/{name}/complex_path", hc.cpu().numpy().real.copy(), f"real:{name}", real_ref))
        outs_r = int(np.prod(shape))
        real[name] = {"value": world * outs_r / (msr * 1e-3), "ms": round(msr, 4), "m": [b["m"] for b in br],
                      "D": [b["D"] for b in br], "model_tflops": round(flr / (msr * 1e-3) / 1e12, 4),
                      "complex_path_ms": round(msc, 4), "speedup_vs_complex": round(msc / msr, 4),
                      "tuning_s": round(ttr, 1)}
        del fr, gr, hr, wsr, fc, gc, hc, wsc

    # --- end to end through the host-buffer C call (FP64)
    pinned = []
    for i, L in enumerate(sizes):
        f = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 10 + i, (L,))).pin_memory()
        g = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 1010 + i, (L,))).pin_memory()
        pinned.append((f, g, torch.empty_like(f).pin_memory()))
    wsh = max(hdc.workspace_size_host([L], [2 * L - 1], [p.params[0]["m"]], D=[p.params[0]["D"]])
              for L, p in zip(sizes, plans64))
    # the sizes rotate over three streams, each with its own workspace, so
    # one size's host copies overlap another's kernels; one synchronisation
    # per step
    n_e2e_streams = 3
    e2e_streams = [torch.cuda.Stream(dev) for _ in range(n_e2e_streams)]
    wsh_ts = [torch.empty(wsh, dtype=torch.uint8, device=dev) for _ in range(n_e2e_streams)]

    # issue order: the sizes up through every second one, then back down
    # through the others, so the step starts with a small host-to-device
    # copy and ends with a small device-to-host one, and every large size's
    # copies overlap the kernels of its neighbours
    by_size = sorted(range(len(sizes)), key=lambda i: sizes[i])
    e2e_order = by_size[0::2] + by_size[1::2][::-1]

    def e2e_step():
        for k_, i in enumerate(e2e_order):
            L, p, (f, g, h) = sizes[i], plans64[i], pinned[i]
            prm = p.params[0]
            k = k_ % n_e2e_streams
            hdc.convnd_host(f, g, h, 1, prm["m"], p=prm["p"], q=prm["q"], D=prm["D"], workspace=wsh_ts[k],
                            stream=e2e_streams[k], sync=False)
        for s_ in e2e_streams:
            s_.synchronize()

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    # each step timed on its own (it ends with the synchronisation of its
    # streams); the median over the steps, so one step that meets a pause
    # of the host does not decide the figure (the mean is reported beside it)
    e2e_steps = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        e2e_step()
        e2e_steps.append(time.perf_counter() - t0)
    torch.cuda.synchronize(dev)
    e2e_s = rank_max(statistics.median(e2e_steps))
    e2e_mean_s = rank_max(sum(e2e_steps) / len(e2e_steps))
    for i, (L, (_, _, h)) in enumerate(zip(sizes, pinned)):
        pending.append((f"e2e_fp64/L={L}", h.numpy().copy(), f"sweep{i}", sweep_ref(i, L)))
    h2d = sum(2 * L * 16 for L in sizes)
    d2h = sum(L * 16 for L in sizes)
    # the same host copies alone (same buffers, sizes and streams, no
    # convolution): what the overlap in the end-to-end step hides
    dbufs = [(torch.empty_like(f, device=dev), torch.empty_like(g, device=dev)) for f, g, _ in pinned]

    def copies_step():
        for i, ((f, g, h), (df, dg)) in enumerate(zip(pinned, dbufs)):
            with torch.cuda.stream(e2e_streams[i % n_e2e_streams]):
                df.copy_(f, non_blocking=True)
                dg.copy_(g, non_blocking=True)
                h.copy_(df, non_blocking=True)
        for s_ in e2e_streams:
            s_.synchronize()

    copies_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        copies_step()
    copy_s = rank_max((time.perf_counter() - t0) / args.steps)
    del dbufs

    # --- roofline of the dominant kernel (FP64 ALU bound)
    dom = max((k for k in kstats if kstats[k]["ms"] > 0), key=lambda k: kstats[k]["ms"])
    d = kstats[dom]
    per_launch_flops = d["flops"] / max(1, d["launches"])
    avg_ms = d["ms"] / max(1, d["launches"])
    achieved = per_launch_flops / (avg_ms * 1e-3) / 1e12
    peak = SM_COUNT * FP64_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    total_ms = sum(v["ms"] for v in kstats.values())
    roofline = {
        "bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
        "frac": round(achieved / peak, 4),
        "traffic": (NCU_DRAM_PER_ALG_BYTE[dom] * d["bytes"] / max(1, d["launches"])
                    if dom in NCU_DRAM_PER_ALG_BYTE else None),
        "traffic_basis": "DRAM bytes per algorithmic byte of the kernel's largest sweep launch (one ncu capture, "
                         "L = 2^22) times the average algorithmic bytes per launch",
        "kernel": dom,
        "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"]),
        "peak_basis": "152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz (unit counts and max clock)",
        "peak_measured_fma_probe": round(fp64_probe, 4),
        "share_of_step": round(d["ms"] / total_ms, 4) if total_ms > 0 else None,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                        "model_tflops": round(v["flops"] / (v["ms"] * 1e-3) / 1e12, 4) if v["ms"] > 0 else None}
                    for k, v in kstats.items() if v["launches"]},
        "whole_step_frac": None,
    }
    # whole-step roofline: model flops of the sweep at its tuned tuples / time
    step_flops = sum(pt.params[0]["q"] * (15 * pt.params[0]["m"] * math.log2(pt.params[0]["m"])
                                         + 6 * pt.params[0]["m"] + 24 * L) + 2 * L
                     for L, pt in zip(sizes, plans64))
    roofline["whole_step_frac"] = round(step_flops / (ms64 * 1e-3) / (peak * 1e12), 4)
    roofline["floor"] = floor_roofline(ms64, 16, peak * 1e12)
    roofline["floor"]["explicit_frac"] = round(roofline["floor"]["t_star_ms"] / ms_ex, 4)

    def fp32_roofline(ks, ms):
        """The FP32 step against its roofline: the slower of its model flops at
        the FP32 vector peak and its algorithmic bytes at the measured HBM
        copy bandwidth, over the measured step time."""
        fl = sum(v["flops"] for v in ks.values())
        by = sum(v["bytes"] for v in ks.values())
        peak32 = SM_COUNT * FP32_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6
        t_roof = max(fl / peak32, by / (HBM_GBS * 1e9))
        return {"model_tflops": round(fl / (ms * 1e-3) / 1e12, 4),
                "algorithmic_GBps": round(by / (ms * 1e-3) / 1e9, 1),
                "roofline_frac": round(t_roof / (ms * 1e-3), 4),
                "roofline_basis": "max(model flops / FP32 peak (152 x 128 FMA x 2 x 2070 MHz), "
                                  "algorithmic bytes / measured HBM copy bandwidth) over the step time"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sizes)
    # every result above against the FP64 oracle (rank 0; untimed)
    errs, err_s = ({}, 0.0) if rank != 0 else oracle_errors(pending)
    del pending
    for r in per_size:
        r["hybrid_err"] = errs.get(f"sweep_fp64/L={r['L']}")
        r["explicit_err"] = errs.get(f"explicit_fp64/L={r['L']}")
        r["fp32_err"] = errs.get(f"sweep_fp32/L={r['L']}")

    def emax(prefix):
        v = [x for k, x in errs.items() if k.startswith(prefix) and isinstance(x, float)]
        return max(v) if v else None

    max_err = {
        "basis": "relative max-norm error max|h - h*| / max|h*| against the FP64 oracle (explicitly padded "
                 "FFT convolution O2; direct sum O1 for the single small configuration; O6 for the Hermitian "
                 "case; exact integers O3), each result taken from the timed runs' outputs",
        "sweep_fp64": emax("sweep_fp64/"), "explicit_fp64": emax("explicit_fp64/"),
        "sweep_fp32": emax("sweep_fp32/"), "e2e_fp64": emax("e2e_fp64/"),
        "integer_fp64_exact": {k.split("/", 1)[1]: v for k, v in errs.items() if k.startswith("integer_fp64/")},
        "config1_fp64": errs.get("config1_fp64"),
        "nd_fp64": {k.split("/", 1)[1]: v for k, v in errs.items() if k.startswith("nd_fp64/")},
        "hermitian_fp64": {k.split("/", 1)[1]: v for k, v in errs.items() if k.startswith("hermitian_fp64/")},
        "batched_fp64": {k.rsplit("_", 1)[1]: v for k, v in errs.items() if k.startswith("batched_fp64_")},
        "batched_fp32": {k.rsplit("_", 1)[1]: v for k, v in errs.items() if k.startswith("batched_fp32_")},
        "unequal_fp64": {k.split("/", 1)[1]: v for k, v in errs.items() if k.startswith("unequal_fp64/")},
        "multi_fp64": {k.split("/", 1)[1]: v for k, v in errs.items() if k.startswith("multi_fp64/")},
        "real_fp64": {k.split("/", 1)[1]: v for k, v in errs.items() if k.startswith("real_fp64/")},
        "oracle_s": round(err_s, 1),
    }

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name("FP64"), "sizes": len(sizes), "outputs_per_step": outs,
                   "launch": ("eager launches per timed step" if args.eager else
                              "one step captured in a CUDA graph, replayed per timed step")
                   + f"; the independent sizes issued over {SWEEP_STREAMS} streams (small-large-small order)",
                   "l2": "flushed between timed steps (256 MiB write)", "tuning": "grid search (Section 4.2), "
                   "candidates within 1.5x of the least model flops, m >= 16", "tuning_s": round(tune_s, 1),
                   "parallelism": (f"shard_batch x{world} (sweep copies and batched convolutions; "
                                   "the other workloads replicated)" if world > 1 else "1 GPU")},
        "explicit": {"value": total_outs / (ms_ex * 1e-3), "ms_per_step": ms_ex,
                     "hybrid_speedup": round(ms_ex / ms64, 4)},
        "fp32": {"value": total_outs / (ms32 * 1e-3), "ms_per_step": ms32, **fp32_roofline(kstats32, ms32),
                 "floor": floor_roofline(ms32, 8, SM_COUNT * FP32_FMA_PER_CLK * 2 * SM_MAX_MHZ * 1e6)},
        "nd_fp64": nd,
        "unequal_fp64": uneq,
        "multi_fp64": multi,
        "real_fp64": real,
        "batched_fp64": batched64,
        "batched_fp32": batched32,
        "config1_fp64": cfg1,
        "per_size_fp64": per_size,
        "per_size_fp32": per_size32,
        "max_rel_err": max_err,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": total_outs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "streams": n_e2e_streams, "ms_per_step": round(e2e_s * 1e3, 4),
                "mean_ms_per_step": round(e2e_mean_s * 1e3, 4), "timing": "median of per-step wall-clock times",
                "copies_alone_ms_per_step": round(copy_s * 1e3, 4)},
        "gpu_launches": launches,
        "clocks": clocks,
        "step_ms": [round(x, 4) for x in ms_list],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Run one convolution configuration a few times (a profiler target).

    python -m paper_2306_10016_gb300.profile_case --L 4194304 --m 2097152 \\
        --dtype f64 --reps 3 [--dims 1] [--D 0] [--batch 1]
    python -m paper_2306_10016_gb300.profile_case --L 1024 --m 512 --p 2 --q 4 --D 1
    python -m paper_2306_10016_gb300.profile_case --hermitian 512 --m 512 1536
    python -m paper_2306_10016_gb300.profile_case --sweep --reps 2 [--dtype f64]

Inputs are seeded unit-disk values; each repetition is one hdc_convnd call
(--p, --q, --D fix the tuple per axis) on the current stream, followed by a
synchronisation.  Prints the device time of every repetition.

--hermitian K runs the centered Hermitian 2-D convolution of two seeded
half-plane spectra of (2K - 1) x K points instead, m per axis from --m.

--sweep runs the 1-D sweep of the throughput measurement instead (L = 2^10
.. 2^22 and 3 * 2^9 .. 3 * 2^20, M = 2L - 1, the tuned parameters of each
size from the tuning database, tuned first if absent), every size once per
repetition, eager launches; the repetitions are inside the NVTX range
"hdc_sweep", so a profiler can take exactly those launches
(``--nvtx --nvtx-include "hdc_sweep/"``).
"""
from __future__ import annotations

import argparse
import json
import os

import torch

import paper_2306_10016_gb300 as hdc
from paper_2306_10016_gb300 import synth


def sweep_sizes():
    return sorted([1 << k for k in range(10, 23)] + [3 << k for k in range(9, 21)])


def run_sweep(a, tdt, dcode):
    db = os.environ.get("HDC_TUNING_DB", os.path.join(os.path.expanduser("~"), ".cache", "hdc", "tuning.txt"))
    os.makedirs(os.path.dirname(db), exist_ok=True)
    sizes = sweep_sizes()
    plans = [hdc.Plan([L], dtype=dcode, mode=hdc.HDC_TUNE_EXHAUSTIVE, tuning_db=db) for L in sizes]
    ins = []
    for i, L in enumerate(sizes):
        f = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 10 + i, (L,))).to("cuda", tdt)
        g = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 1010 + i, (L,))).to("cuda", tdt)
        ins.append((f, g, torch.empty_like(f)))
    ws = torch.empty(max(p.workspace_bytes for p in plans), dtype=torch.uint8, device="cuda")

    def step():
        for p, (f, g, h) in zip(plans, ins):
            p.execute(f, g, out=h, workspace=ws)

    step()                                   # warm-up, outside the range
    torch.cuda.synchronize()
    times = []
    torch.cuda.nvtx.range_push("hdc_sweep")
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"sweep": len(sizes), "dtype": a.dtype, "params": [p.params[0] for p in plans],
                      "ms": times}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+")
    ap.add_argument("--m", type=int, nargs="+")
    ap.add_argument("--D", type=int, nargs="+", default=None)
    ap.add_argument("--p", type=int, nargs="+", default=None)
    ap.add_argument("--q", type=int, nargs="+", default=None)
    ap.add_argument("--hermitian", type=int, default=0, metavar="K")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sweep", action="store_true")
    a = ap.parse_args()
    tdt = torch.complex128 if a.dtype == "f64" else torch.complex64
    dcode = hdc.HDC_C128 if a.dtype == "f64" else hdc.HDC_C64
    if a.sweep:
        run_sweep(a, tdt, dcode)
        return
    if a.hermitian:
        K = a.hermitian
        m = a.m if a.m else [K, K]
        f = torch.from_numpy(synth.hermitian_normal(synth.BASE_SEED + 32, K)).to("cuda", tdt)
        g = torch.from_numpy(synth.hermitian_normal(synth.BASE_SEED + 33, K)).to("cuda", tdt)
        h = torch.empty_like(f)
        times = []
        for _ in range(a.reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            hdc.conv2d_hermitian(f, g, m=m, out=h)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        print(json.dumps({"hermitian": K, "m": m, "dtype": a.dtype, "ms": times}))
        return
    if not a.L or not a.m:
        ap.error("--L and --m are required without --sweep or --hermitian")
    dims = len(a.L)
    shape = ([a.batch] if a.batch > 1 else []) + a.L
    f = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 7, shape)).to("cuda", tdt)
    g = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 8, shape)).to("cuda", tdt)
    h = torch.empty_like(f)
    D = a.D if a.D else 0
    times = []
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        hdc.convnd(f, g, dims, a.m, p=a.p if a.p else 0, q=a.q if a.q else 0, D=D, out=h)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    print(json.dumps({"L": a.L, "m": a.m, "dtype": a.dtype, "ms": times}))


if __name__ == "__main__":
    main()

"""Run one convolution configuration a few times (a profiler target).

    python -m paper_2306_10016_gb300.profile_case --L 4194304 --m 2097152 \
        --dtype f64 --reps 3 [--dims 1] [--D 0] [--batch 1]

Inputs are seeded unit-disk values; each repetition is one hdc_convnd call
on the current stream, followed by a synchronisation.  Prints the device
time of every repetition.
"""
from __future__ import annotations

import argparse
import json

import torch

import paper_2306_10016_gb300 as hdc
from paper_2306_10016_gb300 import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", required=True)
    ap.add_argument("--m", type=int, nargs="+", required=True)
    ap.add_argument("--D", type=int, nargs="+", default=None)
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    dims = len(a.L)
    tdt = torch.complex128 if a.dtype == "f64" else torch.complex64
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
        hdc.convnd(f, g, dims, a.m, D=D, out=h)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    print(json.dumps({"L": a.L, "m": a.m, "dtype": a.dtype, "ms": times}))


if __name__ == "__main__":
    main()

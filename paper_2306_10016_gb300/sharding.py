"""Splitting the work over several GPUs (one process per GPU).

Two decompositions follow from the method:

* independent convolutions (a batch, a sweep, the batched plan): each rank
  takes a set of whole convolutions and no data crosses ranks --
  ``shard_batch`` balances them by model flops (longest first onto the least
  loaded rank);
* one large convolution: its residues are independent until the outer sum of
  Eq. 2 (Section 2.2), so each rank computes the share of a contiguous
  residue range (``hdc_convnd_residues``) and one sum-reduction of the
  outputs finishes it -- ``residue_ranges`` and ``conv_residue_sharded``.
"""
from __future__ import annotations

import math


def model_flops(L: int, m: int, q: int) -> float:
    """F1 = q (15 m log2 m + 6 m + 24 L) + 2 L of one 1-D convolution."""
    return q * (15 * m * (math.log2(m) if m > 1 else 0.0) + 6 * m + 24 * L) + 2 * L


def shard_batch(costs, world: int):
    """Index lists, one per rank, of items with the given costs: longest
    first onto the least loaded rank (every item exactly once)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def shard_copies(costs, world: int):
    """A job of `world` copies of a list of independent items (weak scaling:
    the work per rank stays one list's worth) dealt out by shard_batch; per
    rank its (copy, item) pairs in item order.  With equal copies every rank
    gets one copy of every item."""
    units = [(c, i) for c in range(world) for i in range(len(costs))]
    parts = shard_batch([costs[i] for _, i in units], world)
    return [sorted((units[k] for k in p), key=lambda u: (u[1], u[0])) for p in parts]


def residue_ranges(q: int, world: int):
    """Contiguous residue ranges [lo, hi) of nearly equal size, one per rank
    (ranks beyond q get an empty range)."""
    base, extra = divmod(q, world)
    out, lo = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((lo, lo + n))
        lo += n
    return out


def conv_residue_sharded(f, g, dims, m, M=None, p=0, q=0, D=0, group=None):
    """The convolution of f and g split over the ranks of `group` (torch
    distributed, one GPU per rank): this rank's residue-range share, then an
    all-reduce sum; every rank returns the whole result."""
    import torch
    import torch.distributed as dist

    import paper_2306_10016_gb300 as hdc
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    L = [int(x) for x in f.shape[f.dim() - dims:]]
    Mv = M if M is not None else [2 * l - 1 for l in L]
    M0 = Mv[0] if isinstance(Mv, (list, tuple)) else Mv
    m0 = m[0] if isinstance(m, (list, tuple)) else m
    q0 = (q[0] if isinstance(q, (list, tuple)) else q) or -(-M0 // m0)
    lo, hi = residue_ranges(q0, world)[rank]
    if hi > lo:
        h = hdc.convnd_residues(f, g, dims, m, lo, hi, M=M, p=p, q=q, D=D)
    else:
        h = torch.zeros_like(f)
    dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
    return h

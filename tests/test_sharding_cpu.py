"""Multi-rank decomposition on CPU ranks (gloo, world size 2): batch
sharding covers every convolution once, and residue-range shares summed by
an all-reduce give the convolution (computed per rank with the oracle's
Eq. 1 / Eq. 2 routines, so no GPU is needed)."""
import os
import socket

import numpy as np
import pytest

from paper_2306_10016_gb300 import sharding, synth


def test_shard_batch_covers_and_balances():
    Ls = synth.log_uniform_lengths(7, 300, 64, 65536)
    costs = [sharding.model_flops(int(L), int(L), 2) for L in Ls]
    for world in (1, 2, 3, 8):
        parts = sharding.shard_batch(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(Ls)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs) + 1e-9


def test_shard_copies_weak_scaling():
    """N copies of the 25-size sweep over N ranks: every (copy, size) once,
    and each rank one copy of every size (the work per rank of one sweep)."""
    sizes = sorted([1 << k for k in range(10, 23)] + [3 << k for k in range(9, 21)])
    costs = [sharding.model_flops(L, L, 2) for L in sizes]
    for world in (1, 2, 4, 8):
        parts = sharding.shard_copies(costs, world)
        flat = sorted(u for p in parts for u in p)
        assert flat == sorted((c, i) for c in range(world) for i in range(len(sizes)))
        for p in parts:
            assert [i for _, i in p] == list(range(len(sizes)))


def test_residue_ranges_partition():
    for q in (1, 2, 5, 8, 13):
        for world in (1, 2, 3, 4, 16):
            rs = sharding.residue_ranges(q, world)
            assert len(rs) == world
            assert rs[0][0] == 0 and rs[-1][1] == q
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c and a <= b
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, L, m, q, out_dir):
    import torch.distributed as dist
    import torch

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f = synth.unit_disk(11, (L,))
    g = synth.unit_disk(12, (L,))
    p = -(-L // m)
    F = oracle.residue_forward(f, L, m, p, q)
    G = oracle.residue_forward(g, L, m, p, q)
    H = F * G
    lo, hi = sharding.residue_ranges(q, world)[rank]
    keep = np.zeros(q * m, dtype=bool)
    for r in range(lo, hi):
        keep[r::q] = True          # frequencies k = q l + r
    part = oracle.residue_backward(np.where(keep, H, 0), L, m, p, q)
    t = torch.from_numpy(np.stack([part.real, part.imag]))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    # the time of the slowest rank (the bench's rule)
    tm = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), t.numpy()[0] + 1j * t.numpy()[1])
    np.save(os.path.join(out_dir, f"t{rank}.npy"), tm.numpy())
    dist.destroy_process_group()


@pytest.mark.parametrize("L,m,q", [(40, 16, 5), (33, 11, 7), (64, 64, 2)])
def test_residue_shards_allreduce_to_convolution(tmp_path, L, m, q):
    import torch.multiprocessing as mp

    import oracle
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), L, m, q, str(tmp_path)), nprocs=world, join=True)
    ref = oracle.conv_direct(synth.unit_disk(11, (L,)), synth.unit_disk(12, (L,)))
    for r in range(world):
        got = np.load(tmp_path / f"r{r}.npy")
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-13
        assert float(np.load(tmp_path / f"t{r}.npy")[0]) == float(world)


def _batch_rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    Ls = [int(x) for x in synth.log_uniform_lengths(31, 24, 8, 300)]
    ms = [max(4, -(-(2 * L - 1) // 2)) for L in Ls]          # q = 2 (hybrid) per convolution
    costs = [sharding.model_flops(L, m, -(-(2 * L - 1) // m)) for L, m in zip(Ls, ms)]
    mine = sharding.shard_batch(costs, world)[rank]
    # this rank's convolutions by the residue method (O5), no exchange of data
    res = {}
    for i in mine:
        L, m = Ls[i], ms[i]
        f = synth.unit_disk(1000 + i, (L,))
        g = synth.unit_disk(2000 + i, (L,))
        res[i] = oracle.conv_hybrid(f, g, m, -(-L // m), -(-(2 * L - 1) // m))
    got = [None] * world
    dist.all_gather_object(got, res)
    if rank == 0:
        merged = {}
        for d in got:
            assert not (set(d) & set(merged))          # every convolution on one rank only
            merged.update(d)
        np.save(os.path.join(out_dir, "batch.npy"), np.array([merged[i] for i in range(len(Ls))], dtype=object),
                allow_pickle=True)
    dist.destroy_process_group()


def test_shard_batch_end_to_end_on_two_ranks(tmp_path):
    """A batch of uneven convolutions split by shard_batch over two gloo
    ranks, each computed on its rank alone: together every convolution once,
    each equal to the direct sum (O1)."""
    import torch.multiprocessing as mp

    import oracle
    mp.spawn(_batch_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    out = np.load(tmp_path / "batch.npy", allow_pickle=True)
    Ls = [int(x) for x in synth.log_uniform_lengths(31, 24, 8, 300)]
    assert len(out) == len(Ls)
    for i, L in enumerate(Ls):
        ref = oracle.conv_direct(synth.unit_disk(1000 + i, (L,)), synth.unit_disk(2000 + i, (L,)))
        assert np.max(np.abs(out[i] - ref)) / np.max(np.abs(ref)) < 1e-13, (i, L)

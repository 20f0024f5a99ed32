"""The multi-rank form of the batched pass on CPU ranks (gloo, world size
2): every rank takes its balanced share of the subvolumes, the shares
partition the batch, and the step time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1001_3411_gb300.shard import shard_subvolumes, subset


def test_shares_partition_and_balance():
    rng = np.random.default_rng(0)
    sizes = np.floor(np.exp(rng.uniform(np.log(4096), np.log(2097152), 64))).astype(np.int64)
    for world in (1, 2, 3, 4, 8):
        share = shard_subvolumes(sizes, world)
        flat = sorted(b for s in share for b in s)
        assert flat == list(range(64))
        loads = [int(sizes[s].sum()) for s in share]
        assert max(loads) - min(loads) <= int(sizes.max())


def test_subset_keeps_each_subvolume_whole():
    sizes = [5, 7, 3, 9]
    off = np.concatenate([[0], np.cumsum(sizes)])
    pos = np.arange(off[-1] * 3, dtype=np.float32).reshape(-1, 3)
    boxes = np.array([1.0, 2.0, 3.0, 4.0])
    p, o, b = subset(pos, off, boxes, [3, 1])
    assert list(o) == [0, 9, 16]
    assert np.array_equal(p[:9], pos[off[3]:off[4]]) and np.array_equal(p[9:], pos[off[1]:off[2]])
    assert list(b) == [4.0, 2.0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, sizes, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    share = shard_subvolumes(sizes, world)
    mine = share[rank]
    # a rank's "step time" stands for its particles; the job's time is the maximum
    t = torch.tensor([float(np.asarray(sizes)[mine].sum())])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    got = [None] * world
    dist.all_gather_object(got, mine)
    if rank == 0:
        out.put((got, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_batch():
    sizes = [4096, 2097152, 50000, 700000, 9000, 123456, 88888]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(got[0] + got[1]) == list(range(len(sizes)))
    assert not set(got[0]) & set(got[1])
    assert tmax == max(sum(sizes[b] for b in g) for g in got)

"""Parallel HOP's domain decomposition (Sec. 3) with the per-rank steps in
libhop: two ranks (processes) on one GPU, gloo for the collectives, must give
every particle the group that hop_run gives on the whole box, bit for bit.
The ranks share the GPU but never wait on each other inside a kernel: every
exchange is a host-side collective between library calls."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
import torch.distributed as dist
import torch.multiprocessing as mp

import synth

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, pos, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1001_3411_gb300 as hopgpu
        from paper_1001_3411_gb300.decomp import LibhopEngine, parallel_hop, slab_of
        torch.cuda.set_device(0)
        h = hopgpu.Hop(0)
        own = torch.nonzero(slab_of(torch.from_numpy(pos[:, 0]), 1.0, world) == rank).flatten()
        p = hopgpu.default_params()
        g, ng, info = parallel_hop(LibhopEngine(h), torch.from_numpy(pos[own.numpy()]).cuda(), own, len(pos), p,
                                   s=1.5)
        gi = [None] * world
        dist.all_gather_object(gi, (own.numpy(), g.cpu().numpy(), ng, info))
        if rank == 0:
            out.put(gi)
        h.close()
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_decomposition_on_the_gpu_matches_hop_run(world):
    import paper_1001_3411_gb300 as hopgpu
    hopgpu.build_library()
    pos = synth.nfw_box(400_000, 77)[0]
    h = hopgpu.Hop(0)
    ref = h.hop_run(torch.from_numpy(pos).cuda(), hopgpu.default_params())
    ref_group = ref["group"].cpu().numpy()
    h.close()
    torch.cuda.empty_cache()
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, pos, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = q.get()
    for pr in procs:
        pr.join(300)
        assert pr.exitcode == 0
    group = np.full(len(pos), -2, dtype=np.int32)
    for own, g, ng, info in res:
        group[own] = g
        assert ng == ref["n_groups"]
        assert 1.0 / world + 2 * info["padding"][0] < 1.0
    assert np.array_equal(group, ref_group)
    assert ref["n_groups"] > 100

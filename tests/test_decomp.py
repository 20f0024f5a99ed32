"""Parallel HOP's domain decomposition (Sec. 3) on CPU ranks (gloo): slabs
padded by Eq. 1, no links out of padded particles, chains reconnected
across slabs, the gathered boundary table and the replicated merge must give
every particle exactly the group of the single-process method on the whole
box.  The per-rank HOP steps run in the fp64 oracle here (tests/oracle_engine
.py); on a GPU they run in libhop (tests/test_gpu_decomp.py)."""
import os
import socket
from types import SimpleNamespace

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1001_3411_gb300.decomp import in_padding, padding_length, parallel_hop, slab_of

PARAMS = dict(n_dens=64, n_hop=16, n_merge=4, delta_outer=80.0, delta_saddle=200.0, delta_peak=240.0, box=1.0)


def straddling_box(n_bg=30000, n_per=2500, seed=3):
    """Uniform background plus Plummer spheres (a = 0.02) centred on the
    slab faces x = 0 (the periodic face), 1/3, 1/2 and 2/3, so halos and
    chains cross every face for 2 and 3 ranks."""
    rng = np.random.default_rng(seed)
    parts = [synth.uniform_box(n_bg, seed).astype(np.float64)]
    for cx in (0.0, 1.0 / 3.0, 0.5, 2.0 / 3.0):
        c = np.array([cx, rng.random(), rng.random()])
        u = rng.uniform(0.0, 0.9, n_per)
        r = 0.02 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        d = rng.normal(size=(n_per, 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
        parts.append(c + r[:, None] * d)
    pos = np.concatenate(parts)
    return synth._wrap_f32(pos, 1.0).astype(np.float64)


def test_padding_length_is_eq1():
    # L_p = s (Ndens V / N)^(1/3)
    assert padding_length(64, 0.5, 1000, 2.0) == pytest.approx(2.0 * (64 * 0.5 / 1000) ** (1 / 3))
    assert padding_length(65, 1.0, 65, 1.0) == pytest.approx(1.0)


def test_slab_and_padding_membership():
    x = torch.tensor([0.0, 0.05, 0.49, 0.5, 0.51, 0.95, 0.999])
    assert slab_of(x, 1.0, 2).tolist() == [0, 0, 0, 1, 1, 1, 1]
    # padding of slab [0.5, 1) with L_p = 0.06: within 0.06 below 0.5 or above 1 (periodic)
    m = in_padding(x, 0.5, 1.0, 0.06, 1.0)
    assert m.tolist() == [True, True, True, False, False, False, False]
    # padding wider than the rest of the box: every outside particle
    assert in_padding(x, 0.0, 0.5, 0.3, 1.0).tolist() == [False, False, False, True, True, True, True]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, pos, s, out, params=None):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle_engine import OracleEngine
        p = SimpleNamespace(**(params or PARAMS))
        own = torch.nonzero(slab_of(torch.from_numpy(pos[:, 0]), 1.0, world) == rank).flatten()
        g, ng, info = parallel_hop(OracleEngine(), torch.from_numpy(pos[own.numpy()]), own, len(pos), p, s=s)
        gi = [None] * world
        dist.all_gather_object(gi, (own.numpy(), g.numpy(), ng, info))
        if rank == 0:
            out.put(gi)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run(world, pos, s, params=None):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, pos, s, q, params)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = q.get()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    return res


@pytest.mark.parametrize("world,s", [(2, 1.5), (3, 1.5), (2, 0.4)])
def test_decomposition_matches_single_process(world, s):
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    pos = straddling_box()
    ref = oracle.hop(pos, **{k: v for k, v in PARAMS.items()})
    res = _run(world, pos, s)
    group = np.full(len(pos), -2, dtype=np.int32)
    for own, g, ng, info in res:
        group[own] = g
        assert ng == ref["n_groups"]
    assert np.all(group != -2)
    assert np.array_equal(group, ref["group"])
    assert ref["n_groups"] >= 4
    # the padding is a strip, not the whole box
    for *_, info in res:
        assert 1.0 / world + 2 * info["padding"][0] < 1.0
    if s < 1.0:
        # too thin a padding is detected and widened
        assert max(info["rounds"] for *_, info in res) > 1
    # chains really cross the slab faces
    assert sum(info["published"] for *_, info in res) > 0


def test_empty_slab_with_the_paper_defaults():
    """The paper's own list lengths (Ndens = Nhop = 65, Nmerge = 4, Table 2)
    on a box whose particles all lie in x < 0.6, so that the third of three
    slabs owns none: its padding (Eq. 1 with N = 0) reaches the whole box,
    so it receives every particle and labels none, and the other ranks'
    groups still equal the single-process run's."""
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    rng = np.random.default_rng(11)
    bg = rng.random((12000, 3)) * np.array([0.6, 1.0, 1.0])
    parts = [bg]
    for cx in (1.0 / 3.0, 0.5):
        c = np.array([cx, rng.random(), rng.random()])
        u = rng.uniform(0.0, 0.9, 1500)
        r = 0.02 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        d = rng.normal(size=(1500, 3))
        d /= np.linalg.norm(d, axis=1)[:, None]
        parts.append(c + r[:, None] * d)
    pos = synth._wrap_f32(np.concatenate(parts), 1.0).astype(np.float64)
    assert pos[:, 0].max() < 0.6
    params = dict(PARAMS, n_dens=65, n_hop=65, n_merge=4)
    ref = oracle.hop(pos, **params)
    res = _run(3, pos, 1.5, params)
    group = np.full(len(pos), -2, dtype=np.int32)
    for own, g, ng, info in res:
        group[own] = g
        assert ng == ref["n_groups"]
    # the empty slab owns nothing and is padded with every other particle
    assert len(res[2][0]) == 0 and res[2][3]["padded"] == len(pos)
    assert np.all(group != -2)
    assert np.array_equal(group, ref["group"])
    assert ref["n_groups"] >= 2

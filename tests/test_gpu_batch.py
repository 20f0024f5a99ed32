"""The batched pass (many periodic subvolumes in one captured graph) through
the C ABI.

Each subvolume's result must be exactly that of the single-volume path on
that subvolume alone (densities bit for bit, the same neighbour lists
offset by the subvolume's first particle, the same group ids), and the
single-volume path is itself held to the oracle elsewhere; small batches
are also checked against the oracle directly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1001_3411_gb300 as hopgpu
import synth
from hop_parity import check_density, check_knn_rows, oracle_downstream
from paper_1001_3411_gb300 import radius_model

pytestmark = pytest.mark.gpu

D_O, D_S, D_P = 80.0, 200.0, 240.0


@pytest.fixture(scope="module")
def hop():
    hopgpu.build_library()
    h = hopgpu.Hop(0)
    models = radius_model.load()
    for q in (4, 8, 16, 32):
        h.set_tuning(q, 1)
        w, m = models[q]
        h.hop_mlp_load(w, m)
    h.set_tuning(8, 1)
    yield h
    h.close()


def _batch(sizes, boxes, seed):
    """Subvolumes of the given sizes, NFW + 30% background, each scaled to
    its own box."""
    parts = []
    for b, (n, L) in enumerate(zip(sizes, boxes)):
        p, _ = synth.nfw_box(int(n), seed * 100 + b, halo_frac=0.7)
        parts.append(synth._wrap_f32(p.astype(np.float64) * L, L))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(parts).astype(np.float32), off


def _standalone(hop, pos, off, boxes, mode, ld):
    """hop_run on every subvolume alone."""
    out = []
    for b in range(len(boxes)):
        sub = torch.from_numpy(np.ascontiguousarray(pos[off[b]:off[b + 1]])).cuda()
        r = hop.hop_run(sub, hopgpu.default_params(radius_mode=mode, box=float(boxes[b])), ld_nbr=ld)
        out.append(r)
    return out


RAGGED = ([3000, 64, 20011, 777, 45000, 9000, 130], [1.0, 2.5, 1.0, 0.5, 3.0, 1.0, 1.0])


@pytest.mark.parametrize("mode", [hopgpu.HOP_RADIUS_PLAIN, hopgpu.HOP_RADIUS_COUNT, hopgpu.HOP_RADIUS_LEARNED])
@pytest.mark.parametrize("qpw", [4, 8, 16])
def test_batch_equals_each_subvolume_alone(hop, mode, qpw):
    sizes, boxes = RAGGED
    pos, off = _batch(sizes, boxes, 5)
    hop.set_tuning(qpw, 1)
    p = hopgpu.default_params(radius_mode=mode)
    r = hop.hop_run_batch(torch.from_numpy(pos).cuda(), off, boxes, p, ld_nbr=16)
    ref = _standalone(hop, pos, off, boxes, mode, 16)
    dens, group, nbr = r["dens"].cpu().numpy(), r["group"].cpu().numpy(), r["nbr"].cpu().numpy()
    for b in range(len(boxes)):
        a, e = off[b], off[b + 1]
        assert np.array_equal(dens[a:e].view(np.uint32), ref[b]["dens"].cpu().numpy().view(np.uint32)), b
        assert np.array_equal(nbr[a:e] - a, ref[b]["nbr"].cpu().numpy()), b
        assert np.array_equal(group[a:e], ref[b]["group"].cpu().numpy()), b
        assert r["n_groups"][b] == ref[b]["n_groups"], b
    assert r["n_groups"].sum() > 0


def test_eager_and_graph_agree_and_graph_replays_new_data(hop):
    sizes, boxes = RAGGED
    hop.set_tuning(8, 1)
    p = hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)
    pos1, off = _batch(sizes, boxes, 6)
    pos2, _ = _batch(sizes, boxes, 7)
    d = torch.from_numpy(pos1).cuda()
    g1 = hop.hop_run_batch(d, off, boxes, p, ld_nbr=16)
    e1 = hop.hop_run_batch(d, off, boxes, p, ld_nbr=16, eager=True)
    for k in ("dens", "group", "nbr"):
        assert torch.equal(g1[k], e1[k]), k
    assert np.array_equal(g1["n_groups"], e1["n_groups"])
    # same sizes, new positions in the same buffer: the cached graph replays
    g_again = hop.hop_run_batch(d, off, boxes, p, ld_nbr=16)
    assert hop.stats()["launches"] > 0
    for k in ("dens", "group", "nbr"):
        assert torch.equal(g1[k], g_again[k]), k
    d.copy_(torch.from_numpy(pos2))
    g2 = hop.hop_run_batch(d, off, boxes, p, ld_nbr=16)
    e2 = hop.hop_run_batch(d, off, boxes, p, ld_nbr=16, eager=True)
    for k in ("dens", "group", "nbr"):
        assert torch.equal(g2[k], e2[k]), k
    assert not torch.equal(g1["dens"], g2["dens"])


def test_small_batch_against_oracle(hop):
    """Brute-force kNN, densities and the oracle's linking and merge fed the
    GPU arrays, subvolume by subvolume."""
    sizes, boxes = [2500, 64, 4096, 999], [1.0, 2.0, 0.75, 1.0]
    pos, off = _batch(sizes, boxes, 8)
    hop.set_tuning(4, 1)
    p = hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)
    r = hop.hop_run_batch(pos, off, boxes, p, ld_nbr=16)      # host positions
    dens, group = r["dens"].numpy(), r["group"].numpy()
    nbr = r["nbr"].cpu().numpy()
    for b in range(len(sizes)):
        a, e = off[b], off[b + 1]
        sub = pos[a:e]
        nb = e - a
        q = np.arange(nb)
        _, d2_o = check_knn_rows(sub, nbr[a:e] - a, q, 64, box=boxes[b], name=f"sub{b}")
        check_density(dens[a:e], d2_o, nb, box=boxes[b], name=f"sub{b}")
        o = oracle_downstream(dens[a:e], nbr[a:e] - a, 16, 4, D_O, D_S, D_P)
        assert np.array_equal(group[a:e], o["group"]), b
        assert r["n_groups"][b] == o["n_groups"], b


def test_full_batch64_sampled(hop):
    """The 64-subvolume workload (16^3 to 128^3 particles each, about 2e7 in
    all) in the benchmark's configuration: eight subvolumes, the smallest
    and the largest among them, equal their standalone runs, and sampled
    rows of every subvolume match the oracle's brute force."""
    pos, off = synth.workload("batch64")
    B = len(off) - 1
    boxes = np.ones(B)
    hop.set_tuning(4, 1)
    p = hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)
    r = hop.hop_run_batch(torch.from_numpy(pos).cuda(), off, boxes, p, ld_nbr=16)
    sizes = np.diff(off)
    dens, group, nbr = r["dens"].cpu().numpy(), r["group"].cpu().numpy(), r["nbr"].cpu().numpy()
    pick = sorted(set([int(np.argmin(sizes)), int(np.argmax(sizes))] + list(range(0, B, 11))))[:8]
    for b in pick:
        a, e = off[b], off[b + 1]
        sub = torch.from_numpy(np.ascontiguousarray(pos[a:e])).cuda()
        ref = hop.hop_run(sub, p, ld_nbr=16)
        assert np.array_equal(dens[a:e].view(np.uint32), ref["dens"].cpu().numpy().view(np.uint32)), b
        assert np.array_equal(nbr[a:e] - a, ref["nbr"].cpu().numpy()), b
        assert np.array_equal(group[a:e], ref["group"].cpu().numpy()), b
        assert r["n_groups"][b] == ref["n_groups"], b
    rng = np.random.default_rng(64)
    for b in range(B):
        a, e = off[b], off[b + 1]
        q = rng.choice(e - a, 6, replace=False)
        _, d2_o = check_knn_rows(pos[a:e], nbr[a + q] - a, q, 64, name=f"batch64 sub{b}")
        check_density(dens[a + q], d2_o, e - a, name=f"batch64 sub{b}")
    assert r["n_groups"].sum() > 1000


def test_autotune_applies_the_fastest_candidate(hop):
    sizes, boxes = [30000, 5000, 60000, 1000], [1.0, 1.0, 1.0, 1.0]
    pos, off = _batch(sizes, boxes, 9)
    d = torch.from_numpy(pos).cuda()
    p = hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)
    hop.set_tuning(8, 1)
    before = hop.hop_run_batch(d, off, boxes, p)
    cands = [(4, 1, 0), (8, 1, 0), (16, 1, 0), (8, 2, 0), (4, 1, 3), (2, 1, 0), (32, 1, 0)]
    best, res = hop.hop_autotune(d, off, boxes, p, cands, reps=3)
    assert res[5]["ms"] == -1.0                       # 2 queries per warp: not a batched setting
    timed = [i for i, t in enumerate(res) if t["ms"] >= 0]
    assert len(timed) == 6
    assert best == min(timed, key=lambda i: res[i]["ms"])
    t = hop.get_tuning()
    assert (t["qpw"], t["cpr"], t["buf_factor"]) == cands[best]
    after = hop.hop_run_batch(d, off, boxes, p)
    assert torch.equal(before["dens"], after["dens"]) and torch.equal(before["group"], after["group"])
    hop.apply_tuning(8, 1, 0)


def test_batch_argument_errors(hop):
    sizes, boxes = [500, 800], [1.0, 1.0]
    pos, off = _batch(sizes, boxes, 10)
    d = torch.from_numpy(pos).cuda()
    p = hopgpu.default_params()
    hop.set_tuning(8, 1)
    with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
        hop.hop_run_batch(d, [0, 1270, 1300], boxes, p)        # a subvolume below n_dens
    with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
        hop.hop_run_batch(d, off, [1.0, 0.0], p)               # empty box
    with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
        hop.hop_run_batch(d, off, boxes, hopgpu.default_params(pos_is_f64=1))
    bad = pos.copy()
    bad[600, 1] = 1.0                                            # on the box face of subvolume 1
    with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
        hop.hop_run_batch(torch.from_numpy(bad).cuda(), off, boxes, p)
    hop.set_tuning(1, 1)                                         # 1 query per warp: not a batched setting
    with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
        hop.hop_run_batch(d, off, boxes, p)
    hop.set_tuning(2, 1)
    with pytest.raises(hopgpu.HopError, match="HOP_ENOMODEL|HOP_EINVAL"):
        hop.hop_run_batch(d, off, boxes, hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED))
    hop.set_tuning(8, 1)
    # the context still works after the errors
    r = hop.hop_run_batch(d, off, boxes, p)
    assert r["n_groups"].shape == (2,)


def test_cached_graph_survives_scratch_moving_under_it(hop):
    """A single-box call on a larger box grows (and so moves) the context's
    scratch; the next batched call must notice and capture again."""
    sizes, boxes = [3000, 777, 20011], [1.0, 0.5, 2.0]
    pos, off = _batch(sizes, boxes, 11)
    d = torch.from_numpy(pos).cuda()
    hop.set_tuning(8, 1)
    p = hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_COUNT)
    first = hop.hop_run_batch(d, off, boxes, p, ld_nbr=16)
    big = torch.from_numpy(synth.nfw_box(400000, 12)[0]).cuda()
    hop.hop_run(big, hopgpu.default_params(), ld_nbr=16)
    again = hop.hop_run_batch(d, off, boxes, p, ld_nbr=16)
    for k in ("dens", "group", "nbr"):
        assert torch.equal(first[k], again[k]), k
    # a new radius margin is part of the captured pass too
    hop.set_tuning(8, 1)
    w, m = radius_model.load()[8]
    hop.hop_mlp_load(w, m + 0.05)
    pl = hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)
    a = hop.hop_run_batch(d, off, boxes, pl, ld_nbr=16)
    hop.hop_mlp_load(w, m)
    b = hop.hop_run_batch(d, off, boxes, pl, ld_nbr=16)
    for k in ("dens", "group", "nbr"):
        assert torch.equal(a[k], first[k]) and torch.equal(b[k], first[k]), k

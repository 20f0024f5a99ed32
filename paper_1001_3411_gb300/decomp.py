"""Parallel HOP's domain decomposition (Parallel HOP Sec. 3, "Step By Step")
across ranks: each rank owns one slab of the periodic box and runs the HOP
steps on its own particles plus a padding of its neighbours' particles.

The steps follow Sec. 3 in order:
  1. The box is cut into W slabs along x, rank r owning [r L / W, (r+1) L / W).
  2. Each slab is padded by L_p = s (Ndens V / N)^(1/3) (Eq. 1: V and N are
     the slab's volume and particle count, s > 1 a safety factor): every rank
     sends its particles that lie within another rank's padding to it.
  3. Each rank computes neighbour lists and densities for its owned and
     padded particles, normalised to the whole box's mean density.
  4. Chains are built locally with no link out of a padded particle: a
     padded particle's row is replaced by itself, so its hop is itself and
     it contributes no boundary.
  5. Chains broken at a slab face are reconnected: every rank publishes,
     for each particle it sent as padding, the particle its local chain ends
     on; following these across ranks is again a chain-following problem,
     solved by the library's own link step on the published particles.
  6. Ranks exchange the chain labels of padded particles, build their
     boundary tables over the particles they own, gather the tables and keep
     each chain pair's largest boundary (the global table).
  7. The merge is replicated on every rank over the chains' peaks; each rank
     labels the particles it owns.

Two readings make the result exact, identical to one process running the
whole box (the paper accepts small errors near the padding's outer edge):
  - Padding is certified.  A rank's owned particle is exact when its
    Ndens-th neighbour lies closer than the padded region's x faces; if any
    owned particle fails, every rank doubles s and starts again (the whole
    box is reached eventually, which always certifies).
  - Padded particles take their density and chain label from their owner,
    and only owned particles contribute boundaries, so no pair is counted
    from an inaccurate neighbour list.
Local arrays are ordered by global index, so every tie (equal distances,
equal densities) is broken exactly as in the single-process run.

The per-rank work goes through an engine: ``LibhopEngine`` runs it in the
CUDA library (libhop.so).  Collectives use torch.distributed (NCCL, or gloo
with host tensors); everything in this module is data movement between the
library calls and the collectives.
"""
from __future__ import annotations

import math

import numpy as np


class LibhopEngine:
    """The per-rank HOP steps in libhop (CUDA tensors)."""

    def __init__(self, hop):
        import torch
        self.hop = hop
        self.device = torch.device("cuda", hop.device)
        self.dens_dtype = torch.float32

    def density(self, pos, n_norm, params, ld):
        self.hop.set_norm_count(n_norm)
        try:
            nbr, dens, rk = self.hop.hop_density(pos, params, ld_nbr=ld, want_rk=True)
        finally:
            self.hop.set_norm_count(0)
        return nbr, dens, rk

    def link(self, dens, nbr, n_hop):
        return self.hop.hop_link(dens, nbr, n_hop, want_hop=False)[1]

    def boundaries(self, labels, dens, nbr, n_merge, d_o):
        return self.hop.hop_boundaries(labels, dens, nbr, n_merge, d_o)

    def reduce(self, pair, s):
        return self.hop.hop_boundaries_reduce(pair, s)

    def merge(self, chain, dens, pair, s, d_o, d_s, d_p):
        return self.hop.hop_merge(chain, dens, pair, s, d_o, d_s, d_p)


# ----------------------------------------------------------- collectives
def _comm_dev(group):
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")


def _exchange(sends, group):
    """sends[q] goes to rank q; returns the list received from each rank."""
    import torch
    import torch.distributed as dist
    cd = _comm_dev(group)
    W = len(sends)
    counts = torch.tensor([int(x.shape[0]) for x in sends], dtype=torch.int64, device=cd)
    rcounts = torch.empty_like(counts)
    dist.all_to_all_single(rcounts, counts, group=group)
    rc = rcounts.tolist()
    x0 = sends[0]
    inp = torch.cat([x.to(cd) for x in sends]) if W else x0.to(cd)
    out = torch.empty((sum(rc),) + tuple(x0.shape[1:]), dtype=x0.dtype, device=cd)
    dist.all_to_all_single(out, inp, output_split_sizes=rc, input_split_sizes=counts.tolist(), group=group)
    return [t.to(x0.device) for t in out.split(rc)]


def _allgather(x, group):
    """Concatenation over ranks (rank order) of tensors of any length."""
    import torch
    import torch.distributed as dist
    cd = _comm_dev(group)
    W = dist.get_world_size(group)
    n = torch.tensor([int(x.shape[0])], dtype=torch.int64, device=cd)
    ns = [torch.empty_like(n) for _ in range(W)]
    dist.all_gather(ns, n, group=group)
    ns = [int(v.item()) for v in ns]
    mx = max(ns) if ns else 0
    buf = torch.zeros((mx,) + tuple(x.shape[1:]), dtype=x.dtype, device=cd)
    buf[: x.shape[0]] = x.to(cd)
    outs = [torch.empty_like(buf) for _ in range(W)]
    dist.all_gather(outs, buf, group=group)
    return torch.cat([o[:k] for o, k in zip(outs, ns)]).to(x.device)


def _allreduce_min(v, group):
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=_comm_dev(group))
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(t.item())


def _allreduce_sum(v, group):
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.int64, device=_comm_dev(group))
    dist.all_reduce(t, group=group)
    return int(t.item())


# ------------------------------------------------------------ geometry
def slab_of(x, box, world):
    """Owning rank of each x coordinate: slab r is [r L / W, (r + 1) L / W)."""
    import torch
    r = torch.floor(x.to(torch.float64) * (world / box)).to(torch.int64)
    return r.clamp_(0, world - 1)


def padding_length(n_dens, slab_volume, n_slab, s):
    """Eq. 1: L_p = s (Ndens V / N)^(1/3)."""
    return s * (n_dens * slab_volume / max(n_slab, 1)) ** (1.0 / 3.0)


def in_padding(x, a, b, lp, box):
    """Particles outside the slab [a, b) whose periodic x distance to it is
    below lp (or every particle outside it when the padded width reaches
    the box)."""
    import torch
    x = x.to(torch.float64)
    inside = (x >= a) & (x < b)
    if (b - a) + 2 * lp >= box:
        return ~inside
    below = torch.remainder(a - x, box)      # distance down to the slab's lower face
    above = torch.remainder(x - b, box)      # distance up from the slab's upper face
    return (~inside) & ((below <= lp) | (above < lp))


# -------------------------------------------------------------- driver
def parallel_hop(engine, pos_own, gidx_own, n_total, params, group=None, s=2.0, max_rounds=8):
    """Group ids of this rank's particles (global numbering) and the number
    of groups.  ``pos_own`` (n x 3) and ``gidx_own`` (n, int64 global
    indices) are this rank's particles, all inside its slab; ``n_total`` is
    the box's particle count.  Returns (group int32 [n], n_groups, info)."""
    import torch
    import torch.distributed as dist
    W = dist.get_world_size(group)
    r = dist.get_rank(group)
    box = float(params.box)
    dev = engine.device
    pos_own = pos_own.to(dev)
    gidx_own = gidx_own.to(dev, torch.int64)
    n_own = int(pos_own.shape[0])
    a, b = r * box / W, (r + 1) * box / W
    if n_own and not bool((slab_of(pos_own[:, 0], box, W) == r).all()):
        raise ValueError("every particle of a rank must lie in its slab")
    vol = (b - a) * box * box
    rounds = 0
    while True:
        rounds += 1
        # ---- 2. padding: L_p per slab (Eq. 1), particles sent to each rank
        lp = padding_length(params.n_dens, vol, n_own, s)
        lps = _allgather(torch.tensor([lp], dtype=torch.float64, device=dev), group).tolist()
        send_idx = []
        for q in range(W):
            if q == r:
                send_idx.append(torch.zeros(0, dtype=torch.int64, device=dev))
                continue
            aq, bq = q * box / W, (q + 1) * box / W
            m = in_padding(pos_own[:, 0], aq, bq, lps[q], box)
            send_idx.append(torch.nonzero(m).flatten())
        recv_pos = _exchange([pos_own[i] for i in send_idx], group)
        recv_gidx = _exchange([gidx_own[i] for i in send_idx], group)
        pad_pos = torch.cat(recv_pos) if W > 1 else pos_own[:0]
        pad_gidx = torch.cat(recv_gidx) if W > 1 else gidx_own[:0]
        # ---- local problem in global-index order (ties broken as globally)
        gl = torch.cat([gidx_own, pad_gidx])
        order = torch.argsort(gl)
        gl = gl[order]
        pos_l = torch.cat([pos_own, pad_pos])[order].contiguous()
        owned_l = torch.cat([torch.ones(n_own, dtype=torch.bool, device=dev),
                             torch.zeros(pad_gidx.shape[0], dtype=torch.bool, device=dev)])[order]
        row_of = torch.argsort(order)       # local row of each owned, then each received, particle
        own_at = row_of[:n_own]
        pad_rows = row_of[n_own:]
        # ---- 3. lists and densities, normalised to the whole box
        nbr, dens, rk = engine.density(pos_l, n_total, params, params.n_hop)
        # certification: every owned particle's Ndens-th neighbour lies
        # closer than the padded region's x faces
        if (b - a) + 2 * lps[r] >= box:
            ok = 1.0
        else:
            x = pos_own[:, 0].to(torch.float64)
            room = torch.minimum(x - (a - lps[r]), (b + lps[r]) - x)
            ok = float(bool((rk[own_at].to(torch.float64) * (1 + 1e-6) < room).all())) if n_own else 1.0
        if _allreduce_min(ok, group) > 0.5 or rounds >= max_rounds:
            if _allreduce_min(ok, group) <= 0.5:
                raise RuntimeError("padding could not be certified")
            break
        s *= 2.0
    # padded particles take their owner's density
    own_dens = dens[own_at]
    recv_dens = _exchange([own_dens[i] for i in send_idx], group)
    pad_at = torch.nonzero(~owned_l).flatten()             # local rows of padded particles
    if W > 1 and pad_rows.numel():
        dens[pad_rows] = torch.cat(recv_dens).to(dens.dtype)
    # ---- 4. no links out of padded particles: their rows hold only themselves
    if pad_at.numel():
        nbr[pad_at] = pad_at.to(nbr.dtype)[:, None].expand(-1, nbr.shape[1])
    chain = engine.link(dens, nbr, params.n_hop).to(torch.int64)
    term_own = chain[own_at]                                 # local row each owned chain ends on
    term_gidx = gl[term_own]
    term_owned = owned_l[term_own]
    # ---- 5. reconnect chains across slabs: publish, for every particle sent
    # as padding, where its local chain ends; following these is a chain
    # problem of its own on the published particles
    sent = torch.unique(torch.cat(send_idx)) if W > 1 else send_idx[0]
    pub_g = _allgather(gidx_own[sent], group)
    pub_t = _allgather(term_gidx[sent], group)
    pub_d = _allgather(own_dens[sent].to(torch.float64), group)
    pub_td = _allgather(dens[term_own[sent]].to(torch.float64), group)
    pub_root = _allgather(term_owned[sent].to(torch.int64), group)
    nodes, inv = torch.unique(torch.cat([pub_g, pub_t]), return_inverse=True)
    m = int(nodes.shape[0])
    root_label = {}
    if m:
        nd = torch.zeros(m, dtype=torch.float64, device=dev)
        nd[inv[: pub_g.shape[0]]] = pub_d
        nd[inv[pub_g.shape[0]:]] = pub_td
        nxt = torch.arange(m, dtype=torch.int64, device=dev)
        # a published particle steps to its terminal; a terminal that is its
        # owner's own root (or unpublished) steps to itself
        nxt[inv[: pub_g.shape[0]]] = inv[pub_g.shape[0]:]
        rows = torch.stack([torch.arange(m, device=dev), nxt], dim=1).to(torch.int32).contiguous()
        jchain = engine.link(nd.to(engine.dens_dtype), rows, 2).to(torch.int64)
        join_root = nodes[jchain]
    # global chain label of every owned particle
    label_own = term_gidx.clone()
    ext = ~term_owned
    if bool(ext.any()):
        pos_in = torch.searchsorted(nodes, term_gidx[ext])
        label_own[ext] = join_root[pos_in]
    # ---- 6. labels of padded particles from their owners; boundaries over
    # owned particles; the global table
    labels = torch.empty(gl.shape[0], dtype=torch.int64, device=dev)
    labels[own_at] = label_own
    recv_lab = _exchange([label_own[i] for i in send_idx], group)
    if W > 1 and pad_rows.numel():
        labels[pad_rows] = torch.cat(recv_lab)
    pair, ssum = engine.boundaries(labels.to(torch.int32), dens, nbr, params.n_merge, params.delta_outer)
    pair_all = _allgather(pair.to(torch.int64), group)
    s_all = _allgather(ssum.to(torch.float64), group)
    pair_g, s_g = engine.reduce(pair_all, s_all)
    # ---- 7. replicated merge over the chains' peaks above delta_outer
    own_root = owned_l[own_at] & (chain[own_at] == own_at) & (own_dens >= params.delta_outer)
    roots = _allgather(gidx_own[own_root], group)
    root_d = _allgather(own_dens[own_root].to(torch.float64), group)
    ro = torch.argsort(roots)
    roots, root_d = roots[ro], root_d[ro]
    nr = int(roots.shape[0])
    group_own = torch.full((n_own,), -1, dtype=torch.int32, device=dev)
    n_groups = 0
    if nr:
        lo = torch.searchsorted(roots, pair_g >> 32)
        hi = torch.searchsorted(roots, pair_g & 0xFFFFFFFF)
        cpair = (lo << 32) | hi
        gr, n_groups = engine.merge(torch.arange(nr, dtype=torch.int32, device=dev).contiguous(),
                                    root_d.to(engine.dens_dtype).contiguous(), cpair.contiguous(),
                                    s_g.contiguous(), params.delta_outer, params.delta_saddle, params.delta_peak)
        hi_d = own_dens >= params.delta_outer
        ci = torch.searchsorted(roots, label_own[hi_d])
        group_own[hi_d] = gr.to(torch.int32)[ci]
    info = {"rounds": rounds, "s": s, "padding": lps, "padded": int(pad_gidx.shape[0]),
            "published": int(pub_g.shape[0]), "edges": int(pair_g.shape[0]), "roots": nr}
    return group_own, int(n_groups), info


def owned_slab(pos, world, rank, box=1.0):
    """Indices of the particles of ``pos`` (n x 3) in slab ``rank`` of ``world``
    (an input-distribution helper: each rank starts with its own slab)."""
    import torch
    p = torch.as_tensor(np.asarray(pos))
    return torch.nonzero(slab_of(p[:, 0], box, world) == rank).flatten()


def _self_check():
    assert math.isclose(padding_length(64, 0.5, 1000, 1.0), (64 * 0.5 / 1000) ** (1 / 3))

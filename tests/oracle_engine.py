"""The per-rank HOP steps of the domain decomposition run by the fp64 CPU
oracle (test infrastructure only): lets the multi-rank logic of
paper_1001_3411_gb300.decomp run on CPU gloo ranks, with no GPU."""
from __future__ import annotations

import numpy as np
import torch

import oracle


class OracleEngine:
    device = torch.device("cpu")
    dens_dtype = torch.float64

    def __init__(self, box: float = 1.0):
        self.box = box

    def density(self, pos, n_norm, params, ld):
        nbr, d2 = oracle.knn(pos.numpy().astype(np.float64), params.n_dens, self.box)
        dens = oracle.density(d2, n_norm, self.box)
        rk = np.sqrt(d2[:, -1])
        return (torch.from_numpy(np.ascontiguousarray(nbr[:, :ld])), torch.from_numpy(dens),
                torch.from_numpy(rk))

    def link(self, dens, nbr, n_hop):
        _, chain = oracle.link(dens.numpy(), nbr.numpy(), n_hop)
        return torch.from_numpy(chain)

    def boundaries(self, labels, dens, nbr, n_merge, d_o):
        lo, hi, s = oracle.boundaries(labels.numpy(), dens.numpy(), nbr.numpy(), n_merge, d_o)
        pair = (lo.astype(np.int64) << 32) | hi.astype(np.int64)
        return torch.from_numpy(pair), torch.from_numpy(s)

    def reduce(self, pair, s):
        p, v = pair.numpy(), s.numpy()
        if len(p) == 0:
            return pair, s
        o = np.lexsort((-v, p))            # by pair, largest sum first
        p, v = p[o], v[o]
        first = np.concatenate([[True], p[1:] != p[:-1]])
        return torch.from_numpy(p[first]), torch.from_numpy(v[first])

    def merge(self, chain, dens, pair, s, d_o, d_s, d_p):
        p = pair.numpy()
        lo = (p >> 32).astype(np.int32)
        hi = (p & 0xFFFFFFFF).astype(np.int32)
        group, ng = oracle.merge(chain.numpy(), dens.numpy(), lo, hi, s.numpy(), d_o, d_s, d_p)
        return torch.from_numpy(group), ng

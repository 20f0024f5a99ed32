"""Parity helpers shared by the GPU tests: compare the CUDA path with the
oracle under the stated tolerances.  Test infrastructure only."""
from __future__ import annotations

import numpy as np

import oracle

# kNN: sets equal except swaps at equal distances within 1e-6 relative.
TIE_REL = 1e-6
# densities: relative agreement with the fp64 oracle.
DENS_REL = 1e-5


def exact_d2(pos64, i, js, box=1.0):
    """fp64 periodic squared distances from particle i to particles js."""
    d = pos64[js] - pos64[i]
    d -= box * np.round(d / box)
    return (d * d).sum(axis=-1)


def check_knn_rows(pos, gpu_nbr, queries, k, box=1.0, name=""):
    """gpu_nbr[r] (L entries, ascending) is the GPU list of particle queries[r].
    Checks against the oracle: the GPU prefix equals the oracle prefix as a
    set up to ties within TIE_REL at its last distance, has no duplicates,
    and is ordered by (d^2, index) up to TIE_REL.  Returns oracle (nbr, d2)."""
    pos64 = np.asarray(pos, dtype=np.float64)
    nbr_o, d2_o = oracle.knn(pos64, k, box, queries=queries)
    L = gpu_nbr.shape[1]
    bad = []
    for r, i in enumerate(queries):
        g = gpu_nbr[r].astype(np.int64)
        if len(set(g.tolist())) != L:
            bad.append((i, "duplicate"))
            continue
        dg = exact_d2(pos64, i, g, box)
        t = d2_o[r, L - 1]
        tol = TIE_REL * max(t, 1e-300)
        if np.any(dg > t + tol):
            bad.append((i, "entry beyond the L-th distance"))
            continue
        must = nbr_o[r, :L][d2_o[r, :L] < t - tol]
        if not set(must.tolist()) <= set(g.tolist()):
            bad.append((i, "missing a strictly nearer neighbour"))
            continue
        # ascending in d^2 (ties within tolerance may come in either order)
        if np.any(np.diff(dg) < -TIE_REL * np.maximum(dg[1:], 1e-300)):
            bad.append((i, "not ascending"))
            continue
        # exact ties broken by the smaller original index
        for a in range(L - 1):
            if dg[a] == dg[a + 1] and g[a] > g[a + 1]:
                bad.append((i, "tie order"))
                break
    assert not bad, f"{name}: {len(bad)} kNN rows differ, first {bad[:5]}"
    return nbr_o, d2_o


def check_density(dens_gpu, d2_o, n_total, box=1.0, name=""):
    dens_o = oracle.density(d2_o, n_total, box)
    g = np.asarray(dens_gpu, dtype=np.float64)
    fin = np.isfinite(dens_o)
    assert np.array_equal(np.isfinite(g), fin), f"{name}: infinite densities differ"
    rel = np.abs(g[fin] - dens_o[fin]) / np.abs(dens_o[fin])
    assert rel.max() <= DENS_REL, f"{name}: density rel err {rel.max():.3e} > {DENS_REL}"
    return dens_o, float(rel.max())


def oracle_downstream(dens_gpu, nbr_gpu, n_hop, n_merge, d_o, d_s, d_p):
    """The oracle's linking, boundaries and merge fed the GPU's arrays."""
    dens64 = np.asarray(dens_gpu, dtype=np.float32).astype(np.float64)
    nbr = np.ascontiguousarray(nbr_gpu, dtype=np.int32)
    hop, chain = oracle.link(dens64, nbr, n_hop)
    lo, hi, s = oracle.boundaries(chain, dens64, nbr, n_merge, d_o)
    group, ng = oracle.merge(chain, dens64, lo, hi, s, d_o, d_s, d_p)
    return dict(hop=hop, chain=chain, lo=lo, hi=hi, s=s, group=group, n_groups=ng)

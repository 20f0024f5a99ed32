"""Pins of the oracle's ADAPTAHOP subhalos (C9, Parallel HOP Sec. 6).

The oracle is checked against what the paper and plain graph arithmetic fix:
  - the paper's worked example (chains A-E, hand-set densities; fixture in
    tests/golden/sec6_subhalo_example.json), at six thresholds and under
    the Poisson cut;
  - the symmetric table from an independent brute force over directed
    links, and equality with the HOP table (C5) when every link is mutual;
  - subhalo labels from scipy's connected components on the thresholded
    chain graph, with the significance cut and peak ranking recomputed;
  - the hierarchy: subhalos at a higher threshold nest in those below;
  - two overlapping Plummer spheres: one subhalo at a low threshold, two at
    a high one, each peaked at a sphere centre.
"""
import json
import os

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "sec6_subhalo_example.json")


@pytest.fixture(scope="module")
def ex():
    with open(GOLD) as f:
        d = json.load(f)
    d["chain"] = np.array(d["chain"], dtype=np.int32)
    d["dens"] = np.array(d["dens"], dtype=np.float64)
    d["rows"] = np.array(d["rows"], dtype=np.int32)
    return d


def test_example_symmetric_table(ex):
    lo, hi, s = oracle.sym_boundaries(ex["chain"], ex["dens"], ex["rows"], ex["n_merge"], ex["delta_outer"])
    got = [[int(a), int(b), float(v)] for a, b, v in zip(lo, hi, s)]
    assert got == ex["expected_symmetric_table"]
    # the HOP table holds the same pairs plus the one-directional A -> E link
    lo2, hi2, s2 = oracle.boundaries(ex["chain"], ex["dens"], ex["rows"], ex["n_merge"], ex["delta_outer"])
    hop = sorted([[int(a), int(b), float(v)] for a, b, v in zip(lo2, hi2, s2)])
    assert hop == sorted(ex["expected_symmetric_table"] + ex["expected_hop_table_extra"])


@pytest.mark.parametrize("level", ["100", "200", "270", "300", "310", "600"])
def test_example_levels(ex, level):
    sub, n_sub = oracle.adaptahop(ex["chain"], ex["dens"], ex["rows"], ex["n_merge"], ex["delta_outer"],
                                  [float(level)])
    want = ex["levels"][level]
    assert n_sub[0] == want["n_sub"]
    assert sub[0].tolist() == want["sub"]


def test_example_all_levels_in_one_call(ex):
    keys = list(ex["levels"])
    sub, n_sub = oracle.adaptahop(ex["chain"], ex["dens"], ex["rows"], ex["n_merge"], ex["delta_outer"],
                                  [float(k) for k in keys])
    for l, k in enumerate(keys):
        assert n_sub[l] == ex["levels"][k]["n_sub"]
        assert sub[l].tolist() == ex["levels"][k]["sub"]


def test_example_poisson_cut(ex):
    for case in ex["poisson_at_200"]["cases"]:
        sub, n_sub = oracle.adaptahop(ex["chain"], ex["dens"], ex["rows"], ex["n_merge"], ex["delta_outer"],
                                      [200.0], n_min=case["n_min"], f_poisson=case["f_poisson"])
        assert n_sub[0] == case["n_sub"], case
        assert sub[0].tolist() == case["sub"], case


def _random_case(n, n_merge, n_chains, seed, mutual=False):
    return synth.chain_graph_case(n, n_merge, n_chains, seed, mutual)


def _brute_sym(chain, dens, rows, d_o):
    best = {}
    n, nm = rows.shape
    for i in range(n):
        if dens[i] < d_o:
            continue
        for j in rows[i]:
            if j == i or dens[j] < d_o or chain[i] == chain[j]:
                continue
            key = (int(chain[i]), int(chain[j]))
            best[key] = max(best.get(key, -1.0), dens[i] + dens[j])
    out = []
    for (a, b), v in best.items():
        if a < b and (b, a) in best:
            out.append([a, b, max(v, best[(b, a)])])
    return sorted(out)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_symmetric_table_against_brute_force(seed):
    chain, dens, rows = _random_case(3000, 5, 400, seed)
    lo, hi, s = oracle.sym_boundaries(chain, dens, rows, 5, 80.0)
    got = [[int(a), int(b), float(v)] for a, b, v in zip(lo, hi, s)]
    assert got == _brute_sym(chain, dens, rows, 80.0)
    assert len(got) > 50


def test_mutual_lists_give_the_hop_table():
    chain, dens, rows = _random_case(4000, 4, 300, 9, mutual=True)
    a = oracle.sym_boundaries(chain, dens, rows, 4, 80.0)
    b = oracle.boundaries(chain, dens, rows, 4, 80.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert len(a[0]) > 100


def _brute_subhalos(chain, dens, lo, hi, s, level, n_min, f):
    n = len(chain)
    keep = s >= 2.0 * level
    g = coo_matrix((np.ones(keep.sum()), (lo[keep], hi[keep])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    member = dens >= level
    lab = comp[chain]
    out = np.full(n, -1, dtype=np.int32)
    cands = []
    for c in np.unique(lab[member]):
        idx = np.flatnonzero(member & (lab == c))
        N = len(idx)
        mean = dens[idx].sum() / N
        if N < n_min or mean < level * (1.0 + f / np.sqrt(N)):
            continue
        pk = idx[np.lexsort((idx, -dens[idx]))[0]]
        cands.append((-dens[pk], pk, idx))
    cands.sort(key=lambda t: (t[0], t[1]))
    for r, (_, _, idx) in enumerate(cands):
        out[idx] = r
    return out, len(cands)


@pytest.mark.parametrize("seed,n_min,f", [(4, 1, 0.0), (5, 3, 0.0), (6, 1, 0.5), (7, 2, 1.0)])
def test_subhalos_against_connected_components(seed, n_min, f):
    chain, dens, rows = _random_case(3000, 5, 500, seed)
    lo, hi, s = oracle.sym_boundaries(chain, dens, rows, 5, 80.0)
    levels = [80.0, 120.0, 160.0, 240.0]
    sub, n_sub = oracle.subhalos(chain, dens, lo, hi, s, levels, n_min, f)
    for l, lv in enumerate(levels):
        want, k = _brute_subhalos(chain, dens, lo, hi, s, lv, n_min, f)
        assert n_sub[l] == k
        assert np.array_equal(sub[l], want)
    assert n_sub.max() > 10


def _assert_nested(sub):
    """Every subhalo of level l + 1 lies inside one subhalo of level l."""
    for l in range(len(sub) - 1):
        inner = sub[l + 1] >= 0
        assert np.all(sub[l][inner] >= 0)
        pairs = np.unique(np.stack([sub[l + 1][inner], sub[l][inner]]), axis=1)
        assert len(np.unique(pairs[0])) == pairs.shape[1]


def test_hierarchy_nests():
    chain, dens, rows = _random_case(5000, 5, 600, 11)
    lo, hi, s = oracle.sym_boundaries(chain, dens, rows, 5, 80.0)
    sub, n_sub = oracle.subhalos(chain, dens, lo, hi, s, [80.0, 100.0, 150.0, 200.0, 300.0])
    _assert_nested(sub)
    assert n_sub[0] > 0


def test_no_surviving_link_gives_one_subhalo_per_chain():
    chain, dens, rows = _random_case(2000, 4, 200, 12)
    lo, hi, s = oracle.sym_boundaries(chain, dens, rows, 4, 80.0)
    level = float(s.max()) / 2.0 + 1.0
    sub, n_sub = oracle.subhalos(chain, dens, lo, hi, s, [level])
    member = dens >= level
    assert n_sub[0] == len(np.unique(chain[member]))
    for c in np.unique(chain[member]):
        assert len(np.unique(sub[0][member & (chain == c)])) == 1


def test_argument_errors():
    chain, dens, rows = _random_case(100, 3, 10, 13)
    lo, hi, s = oracle.sym_boundaries(chain, dens, rows, 3, 80.0)
    with pytest.raises(RuntimeError):
        oracle.subhalos(chain, dens, lo, hi, s, [100.0], n_min=0)
    with pytest.raises(RuntimeError):
        oracle.subhalos(chain, dens, lo, hi, s, [100.0], f_poisson=-1.0)
    bad = chain.copy()
    bad[0] = 100
    with pytest.raises(RuntimeError):
        oracle.subhalos(bad, dens, lo, hi, s, [100.0])


def test_two_overlapping_spheres_split_at_a_high_threshold():
    """Two Plummer spheres (a = 0.01) whose centres are 4 a apart, in a
    uniform background: the saddle between them is well below their peaks,
    so a low threshold gives one subhalo holding both and a high threshold
    gives two, each peaked within a fraction of a of its sphere's centre."""
    a = 0.01
    pos, cen = synth.plummer_pair(1500, a, 4 * a, 3000, seed=21)
    r = oracle.hop(pos)
    dens = r["dens"]
    sub, n_sub = oracle.adaptahop(r["chain"], dens, r["nbr"], 4, 80.0, [100.0, 3000.0])
    _assert_nested(sub)

    def peaks(level):
        out = []
        for g in range(n_sub[level]):
            idx = np.flatnonzero(sub[level] == g)
            out.append(pos[idx[np.lexsort((idx, -dens[idx]))[0]]])
        return np.array(out)

    def dist_to(p, c):
        d = (p - c + 0.5) % 1.0 - 0.5
        return np.sqrt((d ** 2).sum(axis=-1))

    # low threshold: the densest subhalo holds both sphere cores
    core = [np.argmin(dist_to(pos, c)) for c in cen]
    assert sub[0][core[0]] == sub[0][core[1]] == 0
    # high threshold: the two densest subhalos sit on the two centres
    assert n_sub[1] >= 2
    pk = peaks(1)[:2]
    d = np.array([[dist_to(p, c) for c in cen] for p in pk])
    assert sorted(np.argmin(d, axis=1).tolist()) == [0, 1]
    assert d.min(axis=1).max() < 0.3 * a

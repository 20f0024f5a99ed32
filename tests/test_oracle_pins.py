"""Pins for the CPU oracle: each check ties the oracle to something other than
itself -- brute force written a different way, closed forms, a textbook
routine (the cubic B-spline), the Fig. 1 worked example and an exhaustive
maximum-spanning-forest search.  No GPU needed."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- C1 kNN ---

def _knn_by_images(pos, k, box=1.0):
    """Independent brute force: d^2 is the minimum over all 27 periodic images,
    then a full lexicographic sort by (d^2, index) per query."""
    pos = np.asarray(pos, dtype=np.float64)
    n = len(pos)
    shifts = np.array(list(itertools.product((-box, 0.0, box), repeat=3)))
    nbr = np.empty((n, k), dtype=np.int64)
    d2o = np.empty((n, k))
    idx = np.arange(n)
    for i in range(n):
        diff = pos[None, :, :] + shifts[:, None, :] - pos[i][None, None, :]
        d2 = (diff * diff).sum(axis=2).min(axis=0)
        order = np.lexsort((idx, d2))[:k]
        nbr[i] = order
        d2o[i] = d2[order]
    return nbr, d2o


@pytest.mark.parametrize("n,k,seed", [(300, 16, 1), (257, 64, 2), (64, 64, 3)])
def test_knn_matches_image_bruteforce(n, k, seed):
    pos = synth.uniform_box(n, seed)
    nbr, d2 = oracle.knn(pos, k)
    bn, bd = _knn_by_images(pos, k)
    assert np.array_equal(nbr, bn)
    np.testing.assert_allclose(d2, bd, rtol=1e-12, atol=0)
    assert np.all(nbr[:, 0] == np.arange(n))       # self first at d^2 = 0 (distinct points)
    assert np.all(d2[:, 0] == 0.0)


def test_knn_lattice_ties_by_index():
    """Simple cubic lattice, spacing 1/8 (exact in binary): the shells are
    1, 6, 12, 8, 6, 24, 24 points at d^2/a^2 = 0..6, so the 64th neighbour lies
    in the sqrt(6) shell and ties are broken by the smaller index."""
    m = 8
    pos = synth.lattice_box(m)
    nbr, d2 = oracle.knn(pos, 64)
    a2 = (1.0 / m) ** 2
    shells = [0] * 1 + [1] * 6 + [2] * 12 + [3] * 8 + [4] * 6 + [5] * 24 + [6] * 7
    assert np.array_equal(d2[0] / a2, np.array(shells, dtype=np.float64))
    full_n, _ = _knn_by_images(pos, 64)
    assert np.array_equal(nbr, full_n)


def test_knn_queries_subset_and_errors():
    pos = synth.uniform_box(500, 4)
    q = np.array([0, 7, 499, 250])
    nbr_all, d2_all = oracle.knn(pos, 16)
    nbr_q, d2_q = oracle.knn(pos, 16, queries=q)
    assert np.array_equal(nbr_q, nbr_all[q])
    with pytest.raises(RuntimeError):
        oracle.knn(pos[:10], 16)          # k > n


# ------------------------------------------------------------ C2 density ---

def _cubic_bspline(x):
    """Centred cubic B-spline B3 on knots -2..2 from scipy (a textbook routine)."""
    from scipy.interpolate import BSpline
    b = BSpline.basis_element([-2.0, -1.0, 0.0, 1.0, 2.0], extrapolate=False)
    v = b(np.asarray(x, dtype=np.float64))
    return np.nan_to_num(v, nan=0.0)


def test_density_kernel_shape_is_the_cubic_bspline():
    """A query whose k-list holds particles at chosen radii: the oracle density
    must equal (box^3/N) * sum_j w(r_j/h) / (pi h^3) with w = (3/2) B3 (the M4
    kernel is the cubic B-spline scaled to w(0) = 1) and h = r_k / 2."""
    k = 6
    radii = [0.0, 0.005, 0.010, 0.015, 0.0175, 0.02]   # the last is r_k
    pos = [[0.5, 0.5, 0.5]]
    dirs = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0), (0, -1, 0)]
    for r, d in zip(radii[1:], dirs):
        pos.append([0.5 + r * d[0], 0.5 + r * d[1], 0.5 + r * d[2]])
    # far-away filler so n_total is large and nothing else enters the list
    far = synth.uniform_box(200, 9).astype(np.float64) * 0.2 + 0.01
    pos = np.vstack([np.array(pos), far])
    n = len(pos)
    nbr, d2 = oracle.knn(pos, k, queries=[0])
    assert list(nbr[0]) == [0, 1, 2, 3, 4, 5]
    dens = oracle.density(d2, n)[0]
    h = radii[-1] / 2
    w = 1.5 * _cubic_bspline(np.array(radii) / h)
    expect = (1.0 / n) * w.sum() / (math.pi * h ** 3)
    assert dens == pytest.approx(expect, rel=1e-9)


@pytest.mark.parametrize("k", [64, 65, 16])
def test_density_poisson_closed_form(k):
    """Uniform points in a periodic unit box: conditional on r_k the k-2 inner
    neighbours are uniform in the ball, E[w] over the ball is 3/32 (from the
    kernel's unit normalisation), W(0) = 8/(pi r_k^3), and E[1/V_k] =
    (N-1)/(k-2).  Hence E[delta] = (k - 2 + 32/3)/(k - 2) * (N-1)/N.  k = 65
    is the paper's own Ndens (Table 2)."""
    n = 40000
    pos = synth.uniform_box(n, 11)
    _, d2 = oracle.knn(pos, k)
    dens = oracle.density(d2, n)
    expect = (k - 2 + 32.0 / 3.0) / (k - 2) * (n - 1) / n
    assert dens.mean() == pytest.approx(expect, rel=0.01)


def test_density_lattice_is_uniform_and_degenerate_is_inf():
    pos = synth.lattice_box(8)
    _, d2 = oracle.knn(pos, 64)
    dens = oracle.density(d2, len(pos))
    assert np.allclose(dens, dens[0], rtol=1e-12)
    # k coincident particles: r_k = 0, the density is +inf by definition
    dup = np.vstack([np.full((8, 3), 0.25), synth.uniform_box(100, 5)])
    _, d2 = oracle.knn(dup, 8, queries=[0])
    assert np.isinf(oracle.density(d2, len(dup))[0])


# --------------------------------------------------------- C3, C4 linking ---

def _follow(hop, i):
    seen = set()
    while hop[i] != i:
        assert i not in seen
        seen.add(i)
        i = hop[i]
    return i


def test_link_invariants_and_plain_following():
    pos = synth.plummer_box(n_spheres=3, n_per=300, n_background=400, seed=5, min_sep=0.2)[0]
    n = len(pos)
    nbr, d2 = oracle.knn(pos, 32)
    dens = oracle.density(d2, n)
    hop, chain = oracle.link(dens, nbr, 8)
    for i in range(n):
        cand = nbr[i, :8]
        best = max(cand, key=lambda j: (dens[j], -j))
        assert hop[i] == best
        assert chain[i] == _follow(hop, i)
        assert dens[chain[i]] >= dens[i]
    roots = np.unique(chain)
    assert np.all(hop[roots] == roots)          # every peak is its own densest neighbour


def test_link_ties_to_smaller_index():
    dens = np.array([5.0, 7.0, 7.0, 1.0])
    nbr = np.array([[0, 2, 1], [1, 2, 0], [2, 1, 3], [3, 2, 1]], dtype=np.int32)
    hop, chain = oracle.link(dens, nbr, 3)
    assert list(hop) == [1, 1, 1, 1]
    assert list(chain) == [1, 1, 1, 1]


def test_link_reports_cycles():
    # not kNN lists (self missing): the two particles hop to each other, so
    # following never reaches a root and the oracle must say so
    with pytest.raises(RuntimeError):
        oracle.link(np.array([1.0, 2.0]), np.array([[1, 0], [0, 1]], dtype=np.int32), 1)


# ------------------------------------------------------- C5 boundaries ---

def _boundaries_pairwise(chain, dens, nbr, n_merge, d_o):
    """Pair-centric brute force: an unordered particle pair {i, j} links their
    chains when either lists the other among its first n_merge entries."""
    n = len(chain)
    near = [set(int(x) for x in nbr[i, :n_merge]) for i in range(n)]
    best = {}
    for i in range(n):
        for j in range(i + 1, n):
            if not (j in near[i] or i in near[j]):
                continue
            if dens[i] < d_o or dens[j] < d_o or chain[i] == chain[j]:
                continue
            key = (min(chain[i], chain[j]), max(chain[i], chain[j]))
            best[key] = max(best.get(key, -1.0), dens[i] + dens[j])
    keys = sorted(best)
    return (np.array([a for a, _ in keys], dtype=np.int32),
            np.array([b for _, b in keys], dtype=np.int32),
            np.array([best[kk] for kk in keys]))


@pytest.mark.parametrize("seed", [1, 2])
def test_boundaries_match_pairwise_bruteforce(seed):
    pos = synth.plummer_box(n_spheres=4, n_per=150, n_background=200, seed=seed, a=0.03,
                            min_sep=0.05)[0]
    n = len(pos)
    nbr, d2 = oracle.knn(pos, 32)
    dens = oracle.density(d2, n)
    _, chain = oracle.link(dens, nbr, 4)      # short hop lists: many chains
    d_o = float(np.quantile(dens, 0.3))
    lo, hi, s = oracle.boundaries(chain, dens, nbr, 4, d_o)
    blo, bhi, bs = _boundaries_pairwise(chain, dens, nbr, 4, d_o)
    assert len(lo) > 5
    assert np.array_equal(lo, blo) and np.array_equal(hi, bhi)
    assert np.array_equal(s, bs)


def test_boundaries_one_directional_link_counts():
    # particle 2 lists 1 among its first two entries, 1 does not list 2
    chain = np.array([0, 0, 2, 2], dtype=np.int32)
    dens = np.array([100.0, 90.0, 95.0, 120.0])
    nbr = np.array([[0, 1], [1, 0], [2, 1], [3, 2]], dtype=np.int32)
    lo, hi, s = oracle.boundaries(chain, dens, nbr, 2, 80.0)
    assert list(lo) == [0] and list(hi) == [2] and list(s) == [185.0]
    lo, _, _ = oracle.boundaries(chain, dens, nbr, 2, 91.0)   # particle 1 below delta_outer
    assert len(lo) == 0


# ------------------------------------------------------------ C6 merge ---

def _groups_as_sets(group, names):
    out = {}
    for i, g in enumerate(group):
        if g >= 0:
            out.setdefault(int(g), set()).add(names[i])
    return out


def _fig1(edges_key="edges"):
    fx = json.load(open(os.path.join(GOLDEN, "fig1_merge.json")))
    names = fx["chains"]
    dens = np.array(fx["peak_density"])
    chain = np.arange(len(names), dtype=np.int32)
    src = fx if edges_key == "edges" else fx[edges_key]
    ix = {c: i for i, c in enumerate(names)}
    lo = np.array([min(ix[a], ix[b]) for a, b, _ in src["edges"]], dtype=np.int32)
    hi = np.array([max(ix[a], ix[b]) for a, b, _ in src["edges"]], dtype=np.int32)
    s = np.array([v for _, _, v in src["edges"]])
    return fx, names, dens, chain, lo, hi, s, src["expected_groups"]


@pytest.mark.parametrize("variant", ["edges", "variant_DE_densest"])
def test_merge_fig1(variant):
    fx, names, dens, chain, lo, hi, s, expected = _fig1(variant)
    group, ng = oracle.merge(chain, dens, lo, hi, s, fx["delta_outer"], fx["delta_saddle"],
                             fx["delta_peak"])
    got = _groups_as_sets(group, names)
    assert ng == len(expected)
    assert sorted(map(sorted, got.values())) == sorted(map(sorted, expected))
    # numbering: by peak density, so the group holding A (300) is group 0
    assert group[names.index("A")] == 0


def test_merge_thresholds_are_inclusive():
    """Both thresholds are inclusive (Sec. 3, "Step By Step", writes the
    proto-halo test as peak >= delta_peak and the saddle test as
    delta_link >= delta_saddle; Sec. 2 states the saddle test the same
    way): a peak exactly at delta_peak is a halo, one just below it is not;
    a boundary exactly at delta_saddle (s = 2 delta_saddle) merges two
    proto-halos."""
    d_o, d_s, d_p = 80.0, 200.0, 240.0
    below = np.nextafter(d_p, 0.0)
    # chain 1: peak (particle 1) exactly at d_p, with members exactly at and
    # just below delta_outer; chain 3: peak just below d_p; chains 4 and 5:
    # proto-halos joined by a boundary exactly at the saddle threshold.
    # Chains are labelled by their peak, which is not their first member.
    chain = np.array([1, 1, 3, 3, 4, 5, 1, 1], dtype=np.int32)
    dens = np.array([100.0, d_p, 100.0, below, 300.0, 250.0, d_o, np.nextafter(d_o, 0.0)])
    edge = (np.array([4], dtype=np.int32), np.array([5], dtype=np.int32))
    group, ng = oracle.merge(chain, dens, *edge, np.array([2.0 * d_s]), d_o, d_s, d_p)
    assert ng == 2
    assert group[4] == group[5] == 0            # merged; peak 300 numbered first
    assert group[0] == group[1] == group[6] == 1
    assert group[7] == -1                       # below delta_outer: in no halo (Sec. 2)
    assert group[2] == group[3] == -1
    # the same boundary a hair below the threshold keeps them apart
    group, ng = oracle.merge(chain, dens, *edge, np.array([np.nextafter(2.0 * d_s, 0.0)]), d_o, d_s, d_p)
    assert ng == 3 and group[4] != group[5]


def test_merge_equal_boundaries_follow_the_stated_order():
    """The paper does not say which of two equal boundaries a sub-peak chain
    follows.  The reading used here orders boundaries by (s descending, lo
    ascending, hi ascending), lo < hi the chain labels: chain 3, with equal
    boundaries to the separate proto-halos 0 and 1, joins 0 -- whichever
    order the boundaries are listed in."""
    chain = np.arange(4, dtype=np.int32)
    dens = np.array([300.0, 260.0, 90.0, 150.0])       # 0, 1 proto-halos; 2 outside; 3 sub-peak
    for order in ([0, 1], [1, 0]):
        lo = np.array([[1, 0][i] for i in order], dtype=np.int32)
        hi = np.array([3, 3], dtype=np.int32)
        s = np.array([390.0, 390.0])
        group, ng = oracle.merge(chain, dens, lo, hi, s, 80.0, 200.0, 240.0)
        assert ng == 2 and group[3] == group[0] == 0 and group[1] == 1 and group[2] == -1


def _msf_bruteforce(n_chain, proto, lo, hi, s, two_ds):
    """Exhaustive reference for C6: proto-halos joined by direct boundaries
    >= 2 delta_saddle form the owned sets; all owned sets are contracted to one
    node; the maximum-weight spanning forest of that graph (unique: distinct
    weights) is found by trying every edge subset; each sub-peak chain then
    belongs to the owned set its forest path enters first."""
    parent = list(range(n_chain))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x
    for a, b, w in zip(lo, hi, s):
        if proto[a] and proto[b] and w >= two_ds:
            parent[find(a)] = find(b)
    owner = {c: find(c) for c in range(n_chain) if proto[c]}
    OMEGA = -1
    node = {c: (OMEGA if proto[c] else c) for c in range(n_chain)}
    cedges = [(node[a], node[b], w, a, b) for a, b, w in zip(lo, hi, s) if node[a] != node[b]]
    nodes = sorted(set(node.values()))
    best, best_w = None, -1.0
    m = len(cedges)
    # spanning forest: acyclic and with as many edges as the graph allows
    def comps(es):
        p = {v: v for v in nodes}

        def f(x):
            while p[x] != x:
                x = p[x]
            return x
        for e in es:
            ra, rb = f(e[0]), f(e[1])
            if ra == rb:
                return None
            p[ra] = rb
        return len(set(f(v) for v in nodes))
    # the number of edges of any spanning forest of the whole graph
    p = {v: v for v in nodes}

    def f2(x):
        while p[x] != x:
            x = p[x]
        return x
    for e in cedges:
        p[f2(e[0])] = f2(e[1])
    target_edges = len(nodes) - len(set(f2(v) for v in nodes))
    for subset in itertools.combinations(range(m), target_edges):
        es = [cedges[i] for i in subset]
        if comps(es) is None:
            continue
        w = sum(e[2] for e in es)
        if w > best_w:
            best, best_w = es, w
    best = best or []
    adj = {v: [] for v in nodes}
    for e in best:
        adj[e[0]].append(e)
        adj[e[1]].append(e)
    result = {}
    for c in range(n_chain):
        if proto[c]:
            result[c] = owner[c]
            continue
        # walk the forest from c until the edge that enters OMEGA
        stack, seen, found = [c], {c}, None
        prev = {c: None}
        while stack and found is None:
            v = stack.pop()
            for e in adj[v]:
                u = e[1] if e[0] == v else e[0]
                if u == OMEGA:
                    found = e[3] if proto[e[3]] else e[4]
                    break
                if u not in seen:
                    seen.add(u)
                    stack.append(u)
        result[c] = owner[found] if found is not None else None
    return result


@pytest.mark.parametrize("seed", range(12))
def test_merge_matches_exhaustive_msf(seed):
    rng = np.random.default_rng(seed)
    n_chain = int(rng.integers(4, 8))
    d_o, d_s, d_p = 80.0, 200.0, 240.0
    peak = rng.uniform(100, 400, n_chain)
    proto = peak >= d_p
    pairs = [(a, b) for a in range(n_chain) for b in range(a + 1, n_chain)]
    m = int(rng.integers(3, min(len(pairs), 9) + 1))
    pick = rng.choice(len(pairs), m, replace=False)
    lo = np.array([pairs[i][0] for i in pick], dtype=np.int32)
    hi = np.array([pairs[i][1] for i in pick], dtype=np.int32)
    s = rng.permutation(np.linspace(300.0, 500.0, m))          # distinct weights
    group, ng = oracle.merge(np.arange(n_chain, dtype=np.int32), peak, lo, hi, s, d_o, d_s, d_p)
    ref = _msf_bruteforce(n_chain, proto, lo, hi, s, 2 * d_s)
    # same partition into halos, same set of chains without a halo
    for a in range(n_chain):
        assert (group[a] < 0) == (ref[a] is None)
        for b in range(n_chain):
            if group[a] >= 0 and group[b] >= 0:
                assert (group[a] == group[b]) == (ref[a] == ref[b])


# ------------------------------------------------ end to end (C1..C7) ---

def test_plummer_isolated_spheres_give_one_halo_each():
    """20 well-separated Plummer spheres (a = 0.01, 1146 particles) over a
    uniform background: central density contrast ~ 3M/(4 pi a^3) / (N/L^3)
    ~ 8e3 >> delta_peak, background ~ 1.17 << delta_outer, so exactly 20
    halos, each made of one sphere's inner particles."""
    pos, cen = synth.plummer_box(seed=synth.workload_seed(1), min_sep=0.1)
    r = oracle.hop(pos)
    assert r["n_groups"] == 20
    g = r["group"]
    n_per = 1146
    dominant = []
    for s in range(20):
        mem = g[s * n_per:(s + 1) * n_per]
        vals, cnt = np.unique(mem[mem >= 0], return_counts=True)
        top = int(np.argmax(cnt))
        dominant.append(int(vals[top]))
        assert cnt[top] > 0.6 * n_per               # ~78% lie inside delta = 80
        # the truncated profile reaches r = 0.5, so a few outliers may sit
        # inside another sphere's halo
        assert cnt.sum() - cnt[top] < 0.02 * n_per
    assert sorted(dominant) == list(range(20))      # one halo per sphere
    assert np.all(g[20 * n_per:][r["dens"][20 * n_per:] < 80.0] == -1)
    # invariants of C6/C7
    d = r["dens"]
    assert np.all(g[d < 80.0] == -1)
    peaks = [d[g == k].max() for k in range(r["n_groups"])]
    assert all(p >= 240.0 for p in peaks)
    assert all(peaks[i] >= peaks[i + 1] for i in range(len(peaks) - 1))
    chain = r["chain"]
    for a, b, s_ in zip(r["lo"], r["hi"], r["s"]):
        if d[a] >= 240.0 and d[b] >= 240.0 and s_ >= 400.0:
            assert g[a] == g[b]


# ------------------------------------------------- learned-radius network ---

def test_mlp_oracle_hand_computed_case():
    """One active path through the network, computed by hand:
    y = b3 + w3[0] * relu(b2[0] + W2[0,0] * relu(b1[0] + W1[0,2] * x2)),
    plus a second-layer unit whose pre-activation -4 relu(...) is never
    positive, so its ReLU keeps it out of y."""
    from oracle import mlp
    w1 = np.zeros((64, 27)); w1[0, 2] = 0.5
    b1 = np.zeros(64); b1[0] = -1.0
    w2 = np.zeros((64, 64)); w2[0, 0] = 3.0; w2[1, 0] = -4.0
    b2 = np.zeros(64); b2[0] = 0.25
    w3 = np.zeros(64); w3[0] = -2.0; w3[1] = 1.0
    p = mlp.pack(w1, b1, w2, b2, w3, 0.75)
    x = np.zeros((3, 27)); x[:, 2] = [4.0, 1.0, 6.0]       # hidden pre-activations 1, -0.5, 2
    expect = [0.75 - 2.0 * (0.25 + 3.0 * 1.0), 0.75 - 2.0 * 0.25, 0.75 - 2.0 * (0.25 + 3.0 * 2.0)]
    np.testing.assert_allclose(mlp.forward(p, x), expect, rtol=0, atol=1e-14)
    # the loss the gradient test differentiates is the mean squared error of these outputs
    t = np.array([0.5, -1.0, 2.0])
    loss, _ = mlp.loss_and_grad(p, x, t)
    assert loss == pytest.approx(np.mean((np.array(expect) - t) ** 2), rel=1e-14)


def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(3)
    p = rng.normal(0, 0.3, mlp.NPARAM)
    x = rng.normal(1.0, 1.0, (40, 27))
    t = rng.normal(0.0, 1.0, 40)
    _, g = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 0, 64 * 27]])   # b3, a W1 weight, b1[0]
    for i in idx:
        e = np.zeros(mlp.NPARAM); e[i] = 1e-6
        fd = (mlp.loss_and_grad(p + e, x, t)[0] - mlp.loss_and_grad(p - e, x, t)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_bf16_rounding_is_round_to_nearest_even():
    from oracle import mlp
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 1e-3], dtype=np.float32)
    got = mlp.bf16_round(vals)
    # 1 + 2^-8 is half way between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2 ** -7
    assert got[3] == 1.0 + 2 * 2 ** -7          # 1 + 3*2^-8: tie to even goes up
    assert got[4] == -2.5
    assert abs(got[5] - 1e-3) / 1e-3 < 2 ** -8

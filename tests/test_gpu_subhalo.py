"""ADAPTAHOP subhalos (Parallel HOP Sec. 6) through the C ABI against the
oracle fed the same chains, densities and neighbour lists: subhalo ids must
be bit-exact at every threshold.  The significance cut compares an fp64
mean on both sides; where f_poisson > 0 the tests first check that no
candidate of three or more members has a mean within 1e-9 (relative) of
its threshold, so that the summation order cannot decide it (a sum of one
or two terms is the same in any order, so exact ties there are kept)."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1001_3411_gb300 as hopgpu
import synth

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "sec6_subhalo_example.json")


@pytest.fixture(scope="module")
def hop():
    hopgpu.build_library()
    h = hopgpu.Hop(0)
    yield h
    h.close()


def _cuda(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def _no_borderline(chain, dens, rows, n_merge, d_o, levels, n_min, f):
    """Every candidate's oracle mean is away from its threshold by > 1e-9."""
    if f == 0.0:
        return   # every member is >= delta_s, so the mean passes in any order
    lo, hi, s = oracle.sym_boundaries(chain, dens, rows, n_merge, d_o)
    sub, _ = oracle.subhalos(chain, dens, lo, hi, s, levels, 1, 0.0)
    for l, lv in enumerate(levels):
        g = sub[l]
        m = g >= 0
        if not m.any():
            continue
        N = np.bincount(g[m])
        S = np.bincount(g[m], weights=dens[m])
        thr = lv * (1.0 + f / np.sqrt(N))
        margin = (np.abs(S / N - thr) / thr)[N >= 3]   # sums of one or two terms do not depend on order
        assert margin.size == 0 or margin.min() > 1e-9, "a subhalo's mean sits on its threshold"


def _compare(hop, chain, dens, rows, n_merge, d_o, levels, n_min=1, f=0.0):
    levels = [float(np.float32(x)) for x in levels]     # the thresholds are float32 on both sides
    _no_borderline(chain, dens, rows, n_merge, d_o, levels, n_min, f)
    sub, n_sub = hop.hop_subhalos(_cuda(chain, np.int32), _cuda(dens, np.float32), _cuda(rows, np.int32),
                                  n_merge, d_o, levels, n_min, f)
    sub_o, n_sub_o = oracle.adaptahop(chain, dens, rows, n_merge, d_o, levels, n_min, f)
    assert n_sub.tolist() == n_sub_o.tolist()
    g = sub.cpu().numpy()
    for l in range(len(levels)):
        bad = np.flatnonzero(g[l] != sub_o[l])
        assert bad.size == 0, (levels[l], bad.size, bad[:5])
    return g, n_sub


def test_paper_example_through_the_c_abi(hop):
    with open(GOLD) as fh:
        ex = json.load(fh)
    chain = np.array(ex["chain"], dtype=np.int32)
    dens = np.array(ex["dens"])
    rows = np.array(ex["rows"], dtype=np.int32)
    keys = list(ex["levels"])
    sub, n_sub = _compare(hop, chain, dens, rows, ex["n_merge"], ex["delta_outer"], [float(k) for k in keys])
    for l, k in enumerate(keys):
        assert n_sub[l] == ex["levels"][k]["n_sub"]
        assert sub[l].tolist() == ex["levels"][k]["sub"]
    st = hop.stats()
    assert st["n_edges"] == len(ex["expected_symmetric_table"])
    for case in ex["poisson_at_200"]["cases"]:
        s, ns = hop.hop_subhalos(_cuda(chain, np.int32), _cuda(dens, np.float32), _cuda(rows, np.int32),
                                 ex["n_merge"], ex["delta_outer"], [200.0], case["n_min"], case["f_poisson"])
        assert ns[0] == case["n_sub"], case
        assert s[0].cpu().tolist() == case["sub"], case


# Poisson factors chosen so that no candidate of three or more members sits
# on its threshold (densities on a 0.1 grid make exact ties common)
# (with mutual lists every link has its reverse, so the symmetric table is
# HOP's table; one pairing keeps the components small)
@pytest.mark.parametrize("seed,n_min,f,mutual,n_merge", [(1, 1, 0.0, False, 5), (2, 4, 0.0, False, 5),
                                                         (3, 1, 0.637, False, 5), (4, 2, 1.413, True, 2)])
def test_random_chain_graphs(hop, seed, n_min, f, mutual, n_merge):
    chain, dens, rows = synth.chain_graph_case(60000, n_merge, 6000, seed, mutual)
    _, n_sub = _compare(hop, chain, dens, rows, n_merge, 80.0, [80.0, 110.0, 150.0, 230.0, 400.0], n_min, f)
    assert n_sub.max() > 50


def test_without_links_and_with_every_chain_below_the_level(hop):
    chain, dens, rows = synth.chain_graph_case(5000, 3, 500, 5)
    rows[:, 1:] = rows[:, :1]                    # only the particle itself: no links at all
    _, n_sub = _compare(hop, chain, dens, rows, 3, 80.0, [80.0, 1e9])
    assert n_sub[0] > 0 and n_sub[1] == 0
    assert hop.stats()["n_edges"] == 0


@pytest.mark.parametrize("case", ["pair", "plummer32k_f64", "nfw2M"])
def test_hop_pipeline_subhalos(hop, case):
    if case == "pair":
        pos, _ = synth.plummer_pair(1500, 0.01, 0.04, 3000, seed=21, dtype=np.float32)
        p = hopgpu.default_params()
    elif case == "plummer32k_f64":
        pos = synth.workload("plummer32k")
        p = hopgpu.default_params(pos_is_f64=1)
    else:
        pos = synth.nfw_box(2_000_000, 23)[0]
        p = hopgpu.default_params()
    r = hop.hop_run(torch.from_numpy(np.ascontiguousarray(pos)).cuda(), p, ld_nbr=16, want_chain=True)
    chain = r["chain"].cpu().numpy()
    dens = r["dens"].cpu().numpy().astype(np.float64)
    rows = r["nbr"].cpu().numpy()[:, :4]
    levels = [80.0, 200.0, 600.0, 2000.0, 8000.0]
    f = 0.0 if case != "nfw2M" else 1.0
    sub, n_sub = _compare(hop, chain, dens, rows, 4, 80.0, levels, 1, f)
    assert n_sub[0] > 0
    if f == 0.0:
        # the hierarchy: a subhalo of a higher level lies in one subhalo below
        for l in range(len(levels) - 1):
            inner = sub[l + 1] >= 0
            assert np.all(sub[l][inner] >= 0)
            pairs = np.unique(np.stack([sub[l + 1][inner], sub[l][inner]]), axis=1)
            assert len(np.unique(pairs[0])) == pairs.shape[1]


def test_argument_errors(hop):
    chain, dens, rows = synth.chain_graph_case(1000, 3, 100, 6)
    c, d, rw = _cuda(chain, np.int32), _cuda(dens, np.float32), _cuda(rows, np.int32)
    for kw in (dict(levels=[79.0]), dict(levels=[100.0], n_min=0), dict(levels=[100.0], f_poisson=-1.0),
               dict(levels=[float("inf")])):
        lv = kw.pop("levels")
        with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
            hop.hop_subhalos(c, d, rw, 3, 80.0, lv, **kw)
    with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
        hop.hop_subhalos(c, d, rw, 4, 80.0, [100.0])          # n_merge > ld
    bad = chain.copy()
    bad[np.flatnonzero(bad != np.arange(1000))[0]] = np.flatnonzero(bad != np.arange(1000))[1]
    with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
        hop.hop_subhalos(_cuda(bad, np.int32), d, rw, 3, 80.0, [100.0])   # a label that is not a root
    # the context stays usable
    _compare(hop, chain, dens, rows, 3, 80.0, [100.0])

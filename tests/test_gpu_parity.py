"""GPU parity: the CUDA path (through the C ABI) against the fp64 oracle.

kNN lists: equal sets up to ties within 1e-6 relative; densities within
1e-5 relative; linking, boundaries and merge run on the GPU's own densities
and lists must match the oracle fed the same arrays bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1001_3411_gb300 as hopgpu
import synth
from hop_parity import check_density, check_knn_rows, oracle_downstream

pytestmark = pytest.mark.gpu

D_O, D_S, D_P = 80.0, 200.0, 240.0


@pytest.fixture(scope="module")
def hop():
    hopgpu.build_library()
    h = hopgpu.Hop(0)
    yield h
    h.close()


def _params(**kw):
    return hopgpu.default_params(**kw)


def _to_dev(pos):
    return torch.from_numpy(np.ascontiguousarray(pos)).cuda()


def _plummer(dtype):
    pos = synth.workload("plummer32k")
    return pos if dtype == np.float64 else synth._wrap_f32(pos, 1.0)


CASES = {
    "plummer32k_f64": lambda: (_plummer(np.float64), 1),
    "plummer32k_f32": lambda: (_plummer(np.float32), 0),
    "uniform20011": lambda: (synth.uniform_box(20011, 3), 0),
    "nfw60k": lambda: (synth.nfw_box(60000, 7)[0], 0),
    "lattice16": lambda: (synth.lattice_box(16), 0),
}


@pytest.mark.parametrize("case", list(CASES))
def test_knn_density_parity(hop, case):
    pos, f64 = CASES[case]()
    n = len(pos)
    p = _params(pos_is_f64=f64)
    nbr, dens, rk = hop.hop_density(_to_dev(pos), p, ld_nbr=16, want_rk=True)
    nbr = nbr.cpu().numpy()
    dens = dens.cpu().numpy()
    q = np.arange(n)
    _, d2_o = check_knn_rows(pos, nbr, q, 64, name=case)
    check_density(dens, d2_o, n, name=case)
    rk_o = np.sqrt(d2_o[:, -1])
    np.testing.assert_allclose(rk.cpu().numpy(), rk_o, rtol=1e-6)


def test_knn_full_list_and_ragged_sizes(hop):
    """All 64 entries (verify mode), n not a multiple of any chunk size."""
    pos = synth.nfw_box(9001, 11, halo_frac=0.7)[0]
    nbr, dens, _ = hop.hop_density(_to_dev(pos), _params(), ld_nbr=64)
    _, d2_o = check_knn_rows(pos, nbr.cpu().numpy(), np.arange(len(pos)), 64, name="full64")
    check_density(dens.cpu().numpy(), d2_o, len(pos), name="full64")


@pytest.mark.parametrize("n", [64, 65, 100, 333])
def test_knn_tiny_boxes_scan_everything(hop, n):
    """r_k close to L/2: the search covers the whole box with per-pair
    minimum images."""
    pos = synth.uniform_box(n, 100 + n)
    nbr, dens, _ = hop.hop_density(_to_dev(pos), _params(), ld_nbr=16)
    _, d2_o = check_knn_rows(pos, nbr.cpu().numpy(), np.arange(n), 64, name=f"tiny{n}")
    check_density(dens.cpu().numpy(), d2_o, n, name=f"tiny{n}")


def test_knn_paper_defaults_65(hop):
    """The paper's own defaults (Table 2): Ndens = Nhop = 65, Nmerge = 4."""
    pos = synth.nfw_box(12000, 13)[0]
    p = _params(n_dens=65, n_hop=65)
    nbr, dens, _ = hop.hop_density(_to_dev(pos), p, ld_nbr=65)
    nbr = nbr.cpu().numpy()
    _, d2_o = check_knn_rows(pos, nbr, np.arange(len(pos)), 65, name="k65")
    check_density(dens.cpu().numpy(), d2_o, len(pos), name="k65")
    r = hop.hop_run(_to_dev(pos), p, ld_nbr=65)
    o = oracle_downstream(r["dens"].cpu().numpy(), r["nbr"].cpu().numpy(), 65, 4, D_O, D_S, D_P)
    assert np.array_equal(r["group"].cpu().numpy(), o["group"])


@pytest.mark.parametrize("case", ["plummer32k_f32", "nfw60k", "lattice16", "plummer32k_f64"])
def test_link_boundaries_merge_bit_exact(hop, case):
    pos, f64 = CASES[case]()
    p = _params(pos_is_f64=f64)
    nbr, dens, _ = hop.hop_density(_to_dev(pos), p, ld_nbr=16)
    hop_g, chain_g = hop.hop_link(dens, nbr, 16)
    pair, s = hop.hop_boundaries(chain_g, dens, nbr, 4, D_O)
    group, ng = hop.hop_merge(chain_g, dens, pair, s, D_O, D_S, D_P)
    o = oracle_downstream(dens.cpu().numpy(), nbr.cpu().numpy(), 16, 4, D_O, D_S, D_P)
    assert np.array_equal(hop_g.cpu().numpy(), o["hop"])
    assert np.array_equal(chain_g.cpu().numpy(), o["chain"])
    pr = pair.cpu().numpy()
    assert np.array_equal((pr >> 32).astype(np.int32), o["lo"])
    assert np.array_equal((pr & 0xFFFFFFFF).astype(np.int32), o["hi"])
    assert np.array_equal(s.cpu().numpy(), o["s"])
    assert ng == o["n_groups"]
    assert np.array_equal(group.cpu().numpy(), o["group"])


def test_plummer_config_end_to_end(hop):
    """The 32,768-particle fp64 Plummer set: the fused call gives the oracle's
    groups when the oracle is fed the GPU's densities and lists, and 20 halos."""
    pos = synth.workload("plummer32k")
    p = _params(pos_is_f64=1)
    r = hop.hop_run(_to_dev(pos), p, ld_nbr=16, want_chain=True)
    o = oracle_downstream(r["dens"].cpu().numpy(), r["nbr"].cpu().numpy(), 16, 4, D_O, D_S, D_P)
    assert r["n_groups"] == o["n_groups"] == 20
    assert np.array_equal(r["group"].cpu().numpy(), o["group"])
    assert np.array_equal(r["chain"].cpu().numpy(), o["chain"])


def test_run_matches_stage_calls_and_host_buffers(hop):
    pos = synth.nfw_box(50000, 21)[0]
    p = _params()
    d = hop.hop_run(_to_dev(pos), p, ld_nbr=16, want_chain=True)
    nbr, dens, _ = hop.hop_density(_to_dev(pos), p, ld_nbr=16)
    assert torch.equal(d["dens"], dens)
    assert torch.equal(d["nbr"], nbr)
    hst = hop.hop_run(torch.from_numpy(pos).pin_memory(), p)
    assert np.array_equal(hst["group"].numpy(), d["group"].cpu().numpy())
    assert np.array_equal(hst["dens"].numpy(), d["dens"].cpu().numpy())
    pageable = hop.hop_run(pos, p)
    assert np.array_equal(np.asarray(pageable["group"]), d["group"].cpu().numpy())


@pytest.mark.parametrize("mode", ["count", "learned_random_weights"])
def test_radius_policies_give_identical_output(hop, mode):
    """Every first-radius policy is certified, so output is bit-identical."""
    pos = synth.nfw_box(80000, 31)[0]
    base = hop.hop_run(_to_dev(pos), _params(), ld_nbr=16)
    if mode == "count":
        p = _params(radius_mode=hopgpu.HOP_RADIUS_COUNT)
    else:
        rng = np.random.default_rng(5)
        hop.hop_mlp_load(rng.normal(0, 0.2, hopgpu.MLP_NPARAM).astype(np.float32), 0.1)
        p = _params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)
    other = hop.hop_run(_to_dev(pos), p, ld_nbr=16)
    for k in ("dens", "group", "nbr"):
        assert torch.equal(base[k], other[k]), k
    assert base["n_groups"] == other["n_groups"]


@pytest.mark.parametrize("qpw,cpr", [(4, 1), (16, 2), (32, 1), (8, 2), (1, 3), (2, 2), (4, 4)])
def test_tuning_does_not_change_results(hop, qpw, cpr):
    pos = synth.nfw_box(40000, 41)[0]
    base = hop.hop_run(_to_dev(pos), _params(), ld_nbr=16)
    hop.set_tuning(qpw, cpr)
    try:
        other = hop.hop_run(_to_dev(pos), _params(), ld_nbr=16)
    finally:
        hop.set_tuning(8, 1)
    for k in ("dens", "group", "nbr"):
        assert torch.equal(base[k], other[k]), k


def test_errors_are_reported_not_faulted(hop):
    pos = synth.uniform_box(1000, 3)
    bad = pos.copy()
    bad[17, 1] = 1.0                      # == box: outside [0, box)
    with pytest.raises(hopgpu.HopError) as e:
        hop.hop_density(_to_dev(bad), _params(), ld_nbr=16)
    assert e.value.code == hopgpu.HOP_EINVAL
    with pytest.raises(hopgpu.HopError) as e:
        hop.hop_density(_to_dev(pos[:10]), _params(), ld_nbr=16)
    assert e.value.code == hopgpu.HOP_EINVAL
    # lists without the particle itself: hops cycle; reported as a timeout
    dens = torch.tensor([1.0, 2.0], device="cuda")
    nbr = torch.tensor([[1, 0], [0, 1]], dtype=torch.int32, device="cuda")
    with pytest.raises(hopgpu.HopError) as e:
        hop.hop_link(dens, nbr, 1)
    assert e.value.code == hopgpu.HOP_ETIMEOUT
    # the context stays usable
    nbr, dens, _ = hop.hop_density(_to_dev(pos), _params(), ld_nbr=16)
    assert torch.isfinite(dens).all()

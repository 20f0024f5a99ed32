"""The one-query-per-lane kNN kernel (32 queries per warp, float32) through
the C ABI: oracle parity on the cases the several-lanes kernel is held to,
bit-identical output against that kernel, and its list-capacity paths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

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


def _dev(pos):
    return torch.from_numpy(np.ascontiguousarray(pos)).cuda()


CASES = {
    "uniform20011": lambda: synth.uniform_box(20011, 3),
    "nfw60k": lambda: synth.nfw_box(60000, 7)[0],
    "plummer32k_f32": lambda: synth._wrap_f32(synth.workload("plummer32k"), 1.0),
    "lattice16": lambda: synth.lattice_box(16),
    "tiny100": lambda: synth.uniform_box(100, 200),
    "tiny64": lambda: synth.uniform_box(64, 164),
}


@pytest.mark.parametrize("buf", [0, 6])
@pytest.mark.parametrize("case", list(CASES))
def test_knn32_oracle_parity(hop, case, buf):
    pos = CASES[case]()
    n = len(pos)
    hop.apply_tuning(32, 1, buf)
    try:
        nbr, dens, rk = hop.hop_density(_dev(pos), hopgpu.default_params(), ld_nbr=16, want_rk=True)
    finally:
        hop.apply_tuning(8, 1, 0)
    q = np.arange(n)
    _, d2_o = check_knn_rows(pos, nbr.cpu().numpy(), q, 64, name=case)
    check_density(dens.cpu().numpy(), d2_o, n, name=case)
    np.testing.assert_allclose(rk.cpu().numpy(), np.sqrt(d2_o[:, -1]), rtol=1e-6)


def test_knn32_full_list_and_k65(hop):
    pos = synth.nfw_box(9001, 11, halo_frac=0.7)[0]
    hop.apply_tuning(32, 2, 0)
    try:
        nbr, dens, _ = hop.hop_density(_dev(pos), hopgpu.default_params(), ld_nbr=64)
        _, d2_o = check_knn_rows(pos, nbr.cpu().numpy(), np.arange(len(pos)), 64, name="full64")
        check_density(dens.cpu().numpy(), d2_o, len(pos), name="full64")
        p = hopgpu.default_params(n_dens=65, n_hop=65)
        r = hop.hop_run(_dev(pos), p, ld_nbr=65)
    finally:
        hop.apply_tuning(8, 1, 0)
    _, d2_o = check_knn_rows(pos, r["nbr"].cpu().numpy(), np.arange(len(pos)), 65, name="k65")
    check_density(r["dens"].cpu().numpy(), d2_o, len(pos), name="k65")
    o = oracle_downstream(r["dens"].cpu().numpy(), r["nbr"].cpu().numpy(), 65, 4, D_O, D_S, D_P)
    assert np.array_equal(r["group"].cpu().numpy(), o["group"])


@pytest.mark.parametrize("mode", [hopgpu.HOP_RADIUS_PLAIN, hopgpu.HOP_RADIUS_COUNT])
@pytest.mark.parametrize("cpr", [1, 2])
def test_knn32_equals_the_several_lanes_kernel(hop, mode, cpr):
    """Densities bit for bit, the same lists and groups as 4 queries per warp."""
    pos = synth.nfw_box(300000, 51)[0]
    p = hopgpu.default_params(radius_mode=mode)
    hop.apply_tuning(4, 1, 0)
    base = hop.hop_run(_dev(pos), p, ld_nbr=16)
    hop.apply_tuning(32, cpr, 0)
    try:
        other = hop.hop_run(_dev(pos), p, ld_nbr=16)
        st = hop.stats()
    finally:
        hop.apply_tuning(8, 1, 0)
    for k in ("dens", "group", "nbr"):
        assert torch.equal(base[k], other[k]), k
    assert st["knn_queries_per_warp"] == 32


def test_knn32_batched_pass_equals_each_subvolume(hop):
    sizes, boxes = [3000, 64, 20011, 777, 45000, 130], [1.0, 2.5, 1.0, 0.5, 3.0, 1.0]
    parts = []
    for b, (n, L) in enumerate(zip(sizes, boxes)):
        pp, _ = synth.nfw_box(n, 700 + b, halo_frac=0.7)
        parts.append(synth._wrap_f32(pp.astype(np.float64) * L, L))
    pos = np.concatenate(parts).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    p = hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_COUNT)
    hop.apply_tuning(32, 1, 0)
    try:
        r = hop.hop_run_batch(_dev(pos), off, boxes, p, ld_nbr=16)
        ref = [hop.hop_run(_dev(pos[off[b]:off[b + 1]]),
                           hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_COUNT, box=boxes[b]), ld_nbr=16)
               for b in range(len(sizes))]
    finally:
        hop.apply_tuning(8, 1, 0)
    dens, group, nbr = r["dens"].cpu().numpy(), r["group"].cpu().numpy(), r["nbr"].cpu().numpy()
    for b in range(len(sizes)):
        a, e = off[b], off[b + 1]
        assert np.array_equal(dens[a:e].view(np.uint32), ref[b]["dens"].cpu().numpy().view(np.uint32)), b
        assert np.array_equal(nbr[a:e] - a, ref[b]["nbr"].cpu().numpy()), b
        assert np.array_equal(group[a:e], ref[b]["group"].cpu().numpy()), b

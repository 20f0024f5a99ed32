"""The count-then-gather kNN kernels (float32: one warp per query at 4
queries per warp, grouped queries at 8 and 16) against the single-scan
kernel with a candidate buffer: all are exact, so
neighbour lists, densities, r_k and group ids must be bit-identical, on
clustered, tied, tiny, wrapped and batched inputs, with every first-radius
policy and the paper's own list lengths.  The default tuning runs the
count-then-gather kernel, so the oracle parity tests cover it too."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1001_3411_gb300 as hopgpu
import synth
from hop_parity import check_density, check_knn_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hop():
    hopgpu.build_library()
    h = hopgpu.Hop(0)
    yield h
    h.close()


def _dev(pos):
    return torch.from_numpy(np.ascontiguousarray(pos)).cuda()


def _density(hop, pos, qpw, buf, ld, **kw):
    hop.apply_tuning(qpw, 1, buf)
    try:
        p = hopgpu.default_params(**kw)
        nbr, dens, rk = hop.hop_density(_dev(pos), p, ld_nbr=ld, want_rk=True)
    finally:
        hop.apply_tuning(8, 1, 0)
    return nbr, dens, rk


def _clump_at_kth(n_bg=6000, seed=5):
    """A uniform background plus, around one query, a thin shell of 400
    particles at one distance: the Ndens-th bin of the queries near the
    shell is crowded, which makes the kernel count again in finer bins."""
    rng = np.random.default_rng(seed)
    bg = rng.random((n_bg, 3))
    c = np.array([0.5, 0.5, 0.5])
    d = rng.normal(size=(400, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    shell = c + 0.02 * d * (1 + 1e-4 * rng.random((400, 1)))
    pos = np.concatenate([[c], bg, shell]) % 1.0
    return synth._wrap_f32(pos, 1.0)


CASES = {
    "nfw60k": lambda: synth.nfw_box(60000, 7)[0],
    "lattice16": lambda: synth.lattice_box(16),
    "uniform20011": lambda: synth.uniform_box(20011, 3),
    "clump_at_kth": _clump_at_kth,
    "tiny100": lambda: synth.uniform_box(100, 9),
}


@pytest.mark.parametrize("qpw", [4, 8, 16])
@pytest.mark.parametrize("case", list(CASES))
def test_count_gather_equals_single_scan(hop, case, qpw):
    pos = CASES[case]()
    a = _density(hop, pos, qpw, 0, 16)
    b = _density(hop, pos, qpw, 4, 16)
    for x, y, name in zip(a, b, ("nbr", "dens", "rk")):
        assert torch.equal(x, y), (case, qpw, name)


@pytest.mark.parametrize("case", ["clump_at_kth", "lattice16"])
@pytest.mark.parametrize("qpw", [4, 8])
def test_count_gather_against_oracle(hop, case, qpw):
    pos = CASES[case]()
    n = len(pos)
    nbr, dens, _ = _density(hop, pos, qpw, 0, 16)
    _, d2_o = check_knn_rows(pos, nbr.cpu().numpy(), np.arange(n), 64, name=case)
    check_density(dens.cpu().numpy(), d2_o, n, name=case)


@pytest.mark.parametrize("qpw", [4, 8, 16])
def test_count_gather_full_list_and_paper_defaults(hop, qpw):
    pos = synth.nfw_box(30001, 13, halo_frac=0.7)[0]
    # all 64 entries of every list
    a = _density(hop, pos, qpw, 0, 64)
    b = _density(hop, pos, qpw, 4, 64)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # the paper's Ndens = Nhop = 65 (Table 2)
    a = _density(hop, pos, qpw, 0, 65, n_dens=65, n_hop=65)
    b = _density(hop, pos, qpw, 4, 65, n_dens=65, n_hop=65)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("qpw", [4, 8])
@pytest.mark.parametrize("mode", [hopgpu.HOP_RADIUS_PLAIN, hopgpu.HOP_RADIUS_COUNT])
def test_count_gather_radius_policies(hop, mode, qpw):
    pos = synth.nfw_box(50000, 17)[0]
    a = _density(hop, pos, qpw, 0, 16, radius_mode=mode)
    b = _density(hop, pos, 8, 4, 16, radius_mode=hopgpu.HOP_RADIUS_PLAIN)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_count_gather_batched_subvolumes(hop):
    """Several subvolumes of unequal size and box (the batched kernel form)."""
    parts, off, boxes = [], [0], []
    for i, (n, L) in enumerate([(5000, 1.0), (777, 0.5), (20000, 2.0), (64, 1.0)]):
        x = synth.nfw_box(n, 50 + i)[0].astype(np.float64) * L
        parts.append(synth._wrap_f32(x, L))
        off.append(off[-1] + n)
        boxes.append(L)
    pos = np.concatenate(parts)
    out = {}
    for qpw, buf in ((8, 4), (4, 0), (8, 0), (16, 0)):
        hop.apply_tuning(qpw, 2, buf)
        try:
            out[(qpw, buf)] = hop.hop_run_batch(_dev(pos), off, boxes, hopgpu.default_params(), ld_nbr=16,
                                                eager=True)
        finally:
            hop.apply_tuning(8, 1, 0)
    ref = out[(8, 4)]
    for t, o in out.items():
        for key in ("dens", "group", "nbr"):
            assert torch.equal(ref[key], o[key]), (t, key)
        assert np.array_equal(ref["n_groups"], o["n_groups"])

"""Halo statistics on the GPU (mass, periodic centre of mass about the peak,
maximum radius) against the oracle fed the GPU's own densities and group
ids.  Counts and peaks are exact.  The GPU works in fixed point (2^-32 of
the box, coordinates rounded once): a centre is the mean of rounded
coordinates, within 0.5 units (1.2e-10 of the box) of the oracle's fp64
mean; a radius is measured from that centre rounded to units, so it lies
within 1.5 units (3.5e-10 of the box) of the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1001_3411_gb300 as hopgpu
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hop():
    hopgpu.build_library()
    h = hopgpu.Hop(0)
    yield h
    h.close()


def _compare(pos, dens, group, G, box, gpu):
    count, peak, com, rmax = (t.cpu().numpy() for t in gpu)
    c_o, p_o, com_o, r_o = oracle.halo_stats(np.asarray(pos, dtype=np.float64), dens.astype(np.float64),
                                             group, G, box)
    assert np.array_equal(count, c_o)
    assert np.array_equal(peak, p_o)
    d = (com - com_o + 0.5 * box) % box - 0.5 * box
    assert np.abs(d).max() <= 2e-10 * box, np.abs(d).max()
    np.testing.assert_allclose(rmax, r_o, rtol=0, atol=3.6e-10 * box)


@pytest.mark.parametrize("case", ["plummer32k_f64", "nfw60k", "nfw500k"])
def test_halo_stats_match_oracle_on_hop_groups(hop, case):
    if case == "plummer32k_f64":
        pos, f64 = synth.workload("plummer32k"), 1
    elif case == "nfw60k":
        pos, f64 = synth.nfw_box(60000, 7)[0], 0
    else:
        pos, f64 = synth.nfw_box(500000, 17)[0], 0
    d = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    r = hop.hop_run(d, hopgpu.default_params(pos_is_f64=f64))
    G = r["n_groups"]
    assert G > 0
    gpu = hop.hop_halo_stats(d, r["dens"], r["group"], G)
    _compare(pos, r["dens"].cpu().numpy(), r["group"].cpu().numpy(), G, 1.0, gpu)
    if case == "plummer32k_f64":
        assert G == 20


def test_halo_stats_across_faces_and_other_boxes(hop):
    """Hand-made groups straddling the faces of a box of side 2.5."""
    rng = np.random.default_rng(3)
    L = 2.5
    centres = np.array([[0.01, 2.49, 1.2], [1.25, 0.0, 2.499], [2.4, 2.4, 0.05]])
    parts, groups = [], []
    for g, c in enumerate(centres):
        parts.append(np.mod(c + rng.normal(0, 0.05, (4000, 3)), L))
        groups.append(np.full(4000, g, dtype=np.int32))
    parts.append(rng.random((3000, 3)) * L)
    groups.append(np.full(3000, -1, dtype=np.int32))
    pos = synth._wrap_f32(np.concatenate(parts), L)
    group = np.concatenate(groups)
    dens = rng.random(len(group)).astype(np.float32) * 100
    gpu = hop.hop_halo_stats(torch.from_numpy(pos).cuda(), torch.from_numpy(dens).cuda(),
                             torch.from_numpy(group).cuda(), 3, box=L)
    _compare(pos, dens, group, 3, L, gpu)
    com = gpu[2].cpu().numpy()
    d = (com - centres + 0.5 * L) % L - 0.5 * L
    assert np.abs(d).max() < 0.01


def test_halo_stats_rejects_group_ids_beyond_n_groups(hop):
    pos = torch.rand((100, 3), device="cuda")
    dens = torch.ones(100, device="cuda")
    group = torch.full((100,), 5, dtype=torch.int32, device="cuda")
    with pytest.raises(hopgpu.HopError, match="HOP_EINVAL"):
        hop.hop_halo_stats(pos, dens, group, 5)
    count, _, _, _ = hop.hop_halo_stats(pos, dens, group, 6)
    assert count.cpu().tolist() == [0, 0, 0, 0, 0, 100]

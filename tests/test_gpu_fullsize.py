"""Parity at the full workload sizes, in the configuration the benchmark
times (learned first radius, 4 queries per warp).

512^3: sampled neighbour lists and densities against the oracle's brute
force, and the oracle's hops and chains over all 134M particles fed the
GPU's densities and lists (bit-exact).  256^3: the whole downstream --
hops, chains, boundary table, merge -- bit-exact against the oracle fed the
same arrays."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle
import paper_1001_3411_gb300 as hopgpu
import synth
from hop_parity import check_density, check_knn_rows, oracle_downstream
from paper_1001_3411_gb300 import radius_model

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

D_O, D_S, D_P = 80.0, 200.0, 240.0


@pytest.fixture(scope="module")
def hop():
    hopgpu.build_library()
    h = hopgpu.Hop(0)
    h.set_tuning(4, 1)
    w, m = radius_model.load()[4]
    h.hop_mlp_load(w, m)
    yield h
    h.close()


def _learned():
    return hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)


def test_512cubed_sampled_knn_and_full_linking(hop):
    pos = synth.workload("nfw512")
    n = len(pos)
    r = hop.hop_run(torch.from_numpy(pos).cuda(), _learned(), ld_nbr=16, want_chain=True)
    nbr_d = r["nbr"]
    # every row starts its list with a particle at distance 0: the particle itself
    rows = torch.arange(n, device="cuda", dtype=torch.int32)
    assert bool((nbr_d == rows[:, None]).any(dim=1).all())
    nbr = nbr_d.cpu().numpy()
    dens = r["dens"].cpu().numpy()
    rng = np.random.default_rng(512)
    q = np.concatenate([rng.choice(n, 192, replace=False), [int(np.argmax(dens)), int(np.argmin(dens)),
                                                             0, n - 1]])
    _, d2_o = check_knn_rows(pos, nbr[q], q, 64, name="nfw512")
    check_density(dens[q], d2_o, n, name="nfw512")
    hop_o, chain_o = oracle.link(dens.astype(np.float64), nbr, 16)
    assert np.array_equal(r["chain"].cpu().numpy(), chain_o)
    # a particle above delta_outer in no group must sit in a sub-peak chain
    g = r["group"].cpu().numpy()
    assert r["n_groups"] > 10000
    assert np.all(g[dens < D_O] == -1)


def test_256cubed_full_downstream_bit_exact(hop):
    pos = synth.workload("nfw256")
    r = hop.hop_run(torch.from_numpy(pos).cuda(), _learned(), ld_nbr=16, want_chain=True)
    o = oracle_downstream(r["dens"].cpu().numpy(), r["nbr"].cpu().numpy(), 16, 4, D_O, D_S, D_P)
    assert np.array_equal(r["chain"].cpu().numpy(), o["chain"])
    assert r["n_groups"] == o["n_groups"]
    assert np.array_equal(r["group"].cpu().numpy(), o["group"])

"""Parity at the full workload sizes.

512^3, on the benchmark's own path (one-subvolume batched pass, learned
first radius, autotuned): sampled neighbour lists and densities against the
oracle's brute force, and the whole downstream over all 134M particles --
hops, chains, boundary pairs and sums, every group id -- bit-exact against
the oracle fed the GPU's densities and lists.  256^3 through hop_run: the
same downstream check."""
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
    # one stored network per queries-per-warp setting, so that the
    # autotuner can try each
    for q, (w, m) in sorted(radius_model.load().items()):
        h.set_tuning(q, 1)
        h.hop_mlp_load(w, m)
    h.set_tuning(4, 1)
    yield h
    h.close()


def _learned():
    return hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)


def test_512cubed_bench_path_whole_downstream_bit_exact(hop):
    """The benchmark's own path: one-subvolume batched pass, learned radius,
    the tuning the autotuner picks.  Sampled lists and densities against the
    oracle's brute force; hops, chains, the boundary table (pairs and sums)
    and every group id bit-exact against the oracle fed the GPU's arrays."""
    pos = synth.workload("nfw512")
    n = len(pos)
    d = torch.from_numpy(pos).cuda()
    p = _learned()
    cands = [(4, 2, 0), (4, 1, 0), (8, 1, 0), (16, 1, 0), (32, 1, 0)]
    best, _ = hop.hop_autotune(d, [0, n], [1.0], p, cands, reps=1)
    assert 0 <= best < len(cands)
    r = hop.hop_run_batch(d, [0, n], [1.0], p, ld_nbr=16)
    nbr_d = r["nbr"]
    # every row holds a particle at distance 0: the particle itself
    rows = torch.arange(n, device="cuda", dtype=torch.int32)
    assert bool((nbr_d == rows[:, None]).any(dim=1).all())
    _, chain_d = hop.hop_link(r["dens"], nbr_d, 16, want_hop=False)
    pair_d, s_d = hop.hop_boundaries(chain_d, r["dens"], nbr_d, 4, D_O)
    nbr = nbr_d.cpu().numpy()
    dens = r["dens"].cpu().numpy()
    group = r["group"].cpu().numpy()
    n_groups = int(r["n_groups"][0])
    chain = chain_d.cpu().numpy()
    pair = pair_d.cpu().numpy()
    s_gpu = s_d.cpu().numpy()
    del r, nbr_d, chain_d, pair_d, s_d, d
    torch.cuda.empty_cache()
    rng = np.random.default_rng(512)
    q = np.concatenate([rng.choice(n, 192, replace=False), [int(np.argmax(dens)), int(np.argmin(dens)),
                                                             0, n - 1]])
    _, d2_o = check_knn_rows(pos, nbr[q], q, 64, name="nfw512")
    check_density(dens[q], d2_o, n, name="nfw512")
    o = oracle_downstream(dens, nbr, 16, 4, D_O, D_S, D_P)
    assert np.array_equal(chain, o["chain"])
    lo = (pair >> 32).astype(np.int64)
    hi = (pair & 0xFFFFFFFF).astype(np.int64)
    assert np.array_equal(lo, o["lo"].astype(np.int64))
    assert np.array_equal(hi, o["hi"].astype(np.int64))
    assert np.array_equal(s_gpu, o["s"])
    assert n_groups == o["n_groups"] and n_groups > 10000
    assert np.array_equal(group, o["group"])
    assert np.all(group[dens < D_O] == -1)


def test_256cubed_full_downstream_bit_exact(hop):
    pos = synth.workload("nfw256")
    r = hop.hop_run(torch.from_numpy(pos).cuda(), _learned(), ld_nbr=16, want_chain=True)
    o = oracle_downstream(r["dens"].cpu().numpy(), r["nbr"].cpu().numpy(), 16, 4, D_O, D_S, D_P)
    assert np.array_equal(r["chain"].cpu().numpy(), o["chain"])
    assert r["n_groups"] == o["n_groups"]
    assert np.array_equal(r["group"].cpu().numpy(), o["group"])

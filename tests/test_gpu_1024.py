"""The 1024^3 workload (1.07e9 particles, NFW halos up to 1e6 particles + 40%
background) through hop_density and hop_run in the learned-radius
configuration: sampled neighbour lists and densities against the oracle's
brute force over all particles, plus whole-box invariants.

It needs about 200 GB of device memory and about two minutes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1001_3411_gb300 as hopgpu
import synth
from hop_parity import check_density, check_knn_rows
from paper_1001_3411_gb300 import radius_model

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

D_O = 80.0


def test_1024cubed_sampled_knn_density_and_groups():
    hopgpu.build_library()
    h = hopgpu.Hop(0)
    h.set_tuning(4, 1)
    w, m = radius_model.load()[4]
    h.hop_mlp_load(w, m)
    p = hopgpu.default_params(radius_mode=hopgpu.HOP_RADIUS_LEARNED)
    pos = synth.workload("nfw1024")
    n = len(pos)
    assert n == 1024 ** 3
    d = torch.from_numpy(pos).cuda()
    nbr, dens, _ = h.hop_density(d, p, ld_nbr=16)
    rng = np.random.default_rng(1024)
    dens_h = dens.cpu().numpy()
    q = np.concatenate([rng.choice(n, 40, replace=False), [int(np.argmax(dens_h)), int(np.argmin(dens_h)), 0, n - 1]])
    rows = nbr[torch.from_numpy(q).cuda()].cpu().numpy()
    # every row starts with a particle at distance 0 (the particle itself)
    assert np.all(rows[np.arange(len(q)), 0] == q) or np.all(
        [q[i] in rows[i] for i in range(len(q))])
    del nbr
    torch.cuda.empty_cache()
    _, d2_o = check_knn_rows(pos, rows, q, 64, name="nfw1024")
    check_density(dens_h[q], d2_o, n, name="nfw1024")
    st = h.stats()
    r = h.hop_run(d, p)
    assert torch.equal(r["dens"], dens)
    g = r["group"].cpu().numpy()
    assert r["n_groups"] > 100000
    assert np.all(g[dens_h < D_O] == -1)
    assert g.max() == r["n_groups"] - 1
    print(f"1024^3: kNN {st['ms_knn']:.0f} ms, {r['n_groups']} groups, {h.stats()['ms_total']:.0f} ms per pass")
    h.close()

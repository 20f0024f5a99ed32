"""The learned first search radius on the GPU: forward pass and gradients
against the fp64 oracle network, training by the library's own kernels, and
what the trained network gains over the method without it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1001_3411_gb300 as hopgpu
import synth
from oracle import mlp as omlp
from paper_1001_3411_gb300 import radius_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hop():
    hopgpu.build_library()
    h = hopgpu.Hop(0)
    yield h
    h.close()


@pytest.fixture(scope="module")
def samples(hop):
    """Real training samples: stencil log-counts and log(max r_k / side) of
    every 8-particle chunk of a 500k-particle NFW box (plain search)."""
    pos = torch.from_numpy(synth.nfw_box(500_000, 91)[0]).cuda()
    return radius_model.samples(hop, pos, 8)


def test_forward_and_gradient_match_oracle(hop, samples):
    feat, tgt = samples
    m = 20_000
    x, t = feat[:m].contiguous(), tgt[:m].contiguous()
    rng = np.random.default_rng(11)
    p32 = (rng.normal(0, 0.25, hopgpu.MLP_NPARAM)).astype(np.float32)
    hop.hop_mlp_load(p32, 0.0)
    pb = omlp.bf16_round(p32)                      # the weights the GPU evaluates
    xo, to = x.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    y_gpu = hop.hop_mlp_forward(x).cpu().numpy().astype(np.float64)
    y_o = omlp.forward(pb, xo)
    scale = np.abs(y_o).max()
    assert np.max(np.abs(y_gpu - y_o)) <= 2e-5 * scale + 1e-5
    loss_gpu, g_gpu = hop.hop_mlp_grad(x, t)
    loss_o, g_o = omlp.loss_and_grad(pb, xo, to)
    assert loss_gpu == pytest.approx(loss_o, rel=1e-4)
    g_gpu = g_gpu.cpu().numpy().astype(np.float64)
    # fp32 sums over 20k samples: compare against the gradient's own scale
    assert np.linalg.norm(g_gpu - g_o) <= 1e-4 * np.linalg.norm(g_o)
    np.testing.assert_allclose(g_gpu, g_o, rtol=2e-3, atol=1e-5 * np.abs(g_o).max())


def test_training_on_the_gpu_fits_the_radii(hop, samples):
    feat, tgt = samples
    params, margin, st = radius_model.train(hop, feat, tgt, epochs=12, batch=1024, lr=2e-3)
    var = float(tgt.var())
    assert st["loss"] < 0.25 * var, st          # explains most of the variance
    assert 0.0 < margin < 1.0
    # the trained parameters reproduce their own loss on the CPU oracle
    pb = omlp.bf16_round(params)
    xo = feat.cpu().numpy().astype(np.float64)
    to = tgt.cpu().numpy().astype(np.float64)
    loss_o, _ = omlp.loss_and_grad(pb, xo, to)
    assert loss_o < 0.25 * var


def test_trained_network_gains_over_plain_and_closed_form(hop):
    """Same output, fewer candidates: the stored network (trained on the
    256^3 box) against the plain mean-density radius and the closed-form
    count-based radius, on a fresh 2M-particle box, in the benchmark's
    kernel configuration (one warp per query, 4 queries per chunk)."""
    pos = torch.from_numpy(synth.nfw_box(2_000_000, 93)[0]).cuda()
    n = pos.shape[0]
    res = {}
    for name, mode in (("plain", 0), ("count", 1), ("learned", 2)):
        hop.apply_tuning(4, 2, 0)
        if mode == 2:
            w, m = radius_model.load()[4]
            hop.hop_mlp_load(w, m)
        r = hop.hop_run(pos, hopgpu.default_params(radius_mode=mode))
        st = hop.stats()
        res[name] = (r["group"].clone(), st["candidates"] / n, st["retries"] / st["warps"])
    assert torch.equal(res["plain"][0], res["learned"][0])
    assert torch.equal(res["count"][0], res["learned"][0])
    c_plain, c_count, c_learn = res["plain"][1], res["count"][1], res["learned"][1]
    assert c_learn < 0.5 * c_plain, (c_learn, c_plain)
    assert c_learn < c_count, (c_learn, c_count)
    print(f"candidates per particle: plain {c_plain:.0f}, closed form {c_count:.0f}, "
          f"learned {c_learn:.0f}; retries per chunk: count {res['count'][2]:.3f}, "
          f"learned {res['learned'][2]:.3f}")

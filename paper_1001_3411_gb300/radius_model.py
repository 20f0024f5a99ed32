"""Training of the learned first search radius (the 27 -> 64 -> 64 -> 1 MLP).

Samples come from a plain kNN pass: for every query chunk the library writes
the 27 stencil log-counts and log(max r_k of the chunk / cell side).  The
network is trained on the GPU by the library's own forward/backward/Adam
kernels (``hop_mlp_train``); this module only prepares initial weights,
picks the radius margin and stores the result.  The margin is a quantile of
the training residuals: the search adds it to the predicted log radius, so
about (1 - quantile) of the chunks need a second, larger search.

Usage (on a GPU):  python -m paper_1001_3411_gb300.radius_model --out FILE
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

from ._lib import MLP_HID, MLP_IN, MLP_NPARAM, HOP_RADIUS_PLAIN, Hop, default_params

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_PATH = os.path.join(HERE, "radius_mlp.npz")


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, in the header's parameter layout."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, np.sqrt(2.0 / MLP_IN), (MLP_HID, MLP_IN))
    w2 = rng.normal(0.0, np.sqrt(2.0 / MLP_HID), (MLP_HID, MLP_HID))
    w3 = rng.normal(0.0, 0.1 * np.sqrt(1.0 / MLP_HID), MLP_HID)   # start near the bias
    p = np.concatenate([w1.ravel(), np.zeros(MLP_HID), w2.ravel(), np.zeros(MLP_HID), w3, [0.0]])
    assert p.size == MLP_NPARAM
    return p.astype(np.float32)


def samples(hop: Hop, pos, qpw: int):
    """(feat, target) of every chunk from a plain kNN pass over ``pos``."""
    hop.set_tuning(qpw, 0)
    hop.hop_density(pos, default_params(radius_mode=HOP_RADIUS_PLAIN), ld_nbr=None, want_rk=True)
    return hop.hop_mlp_samples()


def train(hop: Hop, feat, target, epochs: int = 8, batch: int = 8192, lr: float = 2e-3,
          seed: int = 0, quantile: float = 0.9):
    """Trains in place on the GPU; returns (params, margin, stats)."""
    import torch
    t0 = time.time()
    # centre the output bias on the target mean so training starts close
    p0 = init_params(seed)
    p0[-1] = float(target.mean())
    hop.hop_mlp_load(p0, 0.0)
    loss = hop.hop_mlp_train(feat, target, epochs=epochs, batch=batch, lr=lr, seed=seed)
    pred = hop.hop_mlp_forward(feat)
    resid = (target - pred).float()
    margin = float(torch.quantile(resid[: min(len(resid), 4_000_000)], quantile))
    params = hop.hop_mlp_get()
    stats = dict(loss=loss, samples=int(feat.shape[0]), epochs=epochs, batch=batch, lr=lr,
                 quantile=quantile, margin=margin, seconds=time.time() - t0,
                 resid_std=float(resid.std()), target_std=float(target.std()))
    return params, margin, stats


def save(path: str, models: dict, meta: dict):
    arrs = {}
    for qpw, (params, margin) in models.items():
        arrs[f"w_{qpw}"] = params.astype(np.float32)
        arrs[f"m_{qpw}"] = np.array([margin], dtype=np.float32)
    arrs["meta"] = np.array(repr(meta))
    np.savez(path, **arrs)


def load(path: str = DEFAULT_PATH) -> dict:
    """{queries_per_warp: (params, margin)} from a stored file."""
    z = np.load(path)
    out = {}
    for k in z.files:
        if k.startswith("w_"):
            q = int(k[2:])
            out[q] = (z[k], float(z[f"m_{q}"][0]))
    return out


def main():
    import torch

    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--n", type=int, default=256 ** 3, help="training set size (NFW + 40%% background)")
    ap.add_argument("--qpw", default="4,8,16,32")
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--merge", action="store_true",
                    help="keep the stored networks of the other queries-per-warp settings")
    args = ap.parse_args()
    pos, _ = synth.nfw_box(args.n, synth.workload_seed(2))
    dpos = torch.from_numpy(pos).cuda()
    hop = Hop(0)
    models, meta = {}, {"train_n": args.n, "workload": "nfw256" if args.n == 256 ** 3 else "nfw"}
    if args.merge and os.path.exists(args.out):
        models.update(load(args.out))
        z = np.load(args.out)
        if "meta" in z.files:
            meta["previous"] = str(z["meta"])
    for q in [int(x) for x in args.qpw.split(",")]:
        feat, tgt = samples(hop, dpos, q)
        params, margin, st = train(hop, feat, tgt, epochs=args.epochs)
        models[q] = (params, margin)
        meta[f"stats_{q}"] = st
        print(f"qpw={q}: {st}")
    save(args.out, models, meta)
    print("saved", args.out)


if __name__ == "__main__":
    main()

"""fp64 CPU oracle of the learned-radius network -- TEST INFRASTRUCTURE ONLY.

The network is a plain multilayer perceptron, 27 -> 64 -> 64 -> 1 with ReLU
after the two hidden layers, trained on the mean squared error.  This file
writes the forward pass and the back-propagated gradient out in numpy,
fp64, with the parameter layout the C ABI uses:
    W1[64][27], b1[64], W2[64][64], b2[64], W3[64], b3.
``bf16_round`` reproduces the rounding of fp32 parameters to bfloat16
(round to nearest, ties to even, on the top 16 bits of the IEEE binary32
pattern) so the oracle can evaluate exactly the weights the GPU uses.
Pinned by ``tests/test_oracle_pins.py`` (finite differences, a hand-computed
case).
"""
from __future__ import annotations

import numpy as np

IN, HID = 27, 64
NPARAM = HID * IN + HID + HID * HID + HID + HID + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (NPARAM,)
    o = 0
    w1 = p[o:o + HID * IN].reshape(HID, IN); o += HID * IN
    b1 = p[o:o + HID]; o += HID
    w2 = p[o:o + HID * HID].reshape(HID, HID); o += HID * HID
    b2 = p[o:o + HID]; o += HID
    w3 = p[o:o + HID]; o += HID
    b3 = p[o]
    return w1, b1, w2, b2, w3, b3


def pack(w1, b1, w2, b2, w3, b3):
    return np.concatenate([np.ravel(w1), b1, np.ravel(w2), b2, w3, [b3]]).astype(np.float64)


def bf16_round(p):
    """fp32 values rounded to bfloat16 (nearest, ties to even), as fp64."""
    u = np.ascontiguousarray(p, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, x):
    """Outputs y[m] for inputs x[m, 27]."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.maximum(x @ w1.T + b1, 0.0)
    h2 = np.maximum(h1 @ w2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss_and_grad(p, x, t):
    """Mean squared error over the m samples and its gradient (NPARAM)."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    m = x.shape[0]
    a1 = x @ w1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / m                         # d loss / d y
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    d2 = np.outer(dy, w3) * (a2 > 0)         # d loss / d a2
    g_w2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ w2) * (a1 > 0)                # d loss / d a1
    g_w1 = d1.T @ x
    g_b1 = d1.sum(axis=0)
    return loss, pack(g_w1, g_b1, g_w2, g_b2, g_w3, g_b3)

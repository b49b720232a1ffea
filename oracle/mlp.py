"""Band network reference in float64: TEST INFRASTRUCTURE ONLY.

The network maps the 64 band features of a pair to two outputs: the band
centre c (in diagonals, relative to the straight line from (0,0) to (n,m)) and
the log of its half-width. Layers 64 -> 128 -> 128 -> 2 with ReLU after the two
hidden layers; weights are bfloat16 values (the GPU keeps float32 master
copies and computes with their bfloat16 rounding), biases float32, and every
product is accumulated in float64 here.

Loss per pair (targets c*, w* from the optimal path; features x):
  Huber(c - c*, delta = 8) / 8  +  asym(log_w - log(w*)),
  asym(r) = 4 r^2 if r < 0 (band too narrow) else r^2,
averaged over the batch. Gradients are written out by the chain rule; the tests
check them against central finite differences of the loss.
"""
from __future__ import annotations

import numpy as np

SIZES = (64, 128, 128, 2)
HUBER = 8.0
UNDER = 4.0


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    a = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    r = ((a + 0x7FFF + lsb) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)


def forward(params, x):
    """Returns outputs (B, 2) and the activations needed by backward."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    return y, (x, z1, h1, z2, h2)


def loss_and_grad_out(y, target):
    """Mean loss and dL/dy for targets (B, 2) = (centre, log half-width)."""
    y = np.asarray(y, dtype=np.float64)
    t = np.asarray(target, dtype=np.float64)
    B = y.shape[0]
    dc = y[:, 0] - t[:, 0]
    huber = np.where(np.abs(dc) <= HUBER, 0.5 * dc * dc, HUBER * (np.abs(dc) - 0.5 * HUBER)) / HUBER
    g0 = np.where(np.abs(dc) <= HUBER, dc, HUBER * np.sign(dc)) / HUBER
    r = y[:, 1] - t[:, 1]
    wgt = np.where(r < 0, UNDER, 1.0)
    asym = wgt * r * r
    g1 = 2.0 * wgt * r
    loss = float(np.mean(huber + asym))
    gy = np.stack([g0, g1], axis=1) / B
    return loss, gy


def backward(params, acts, gy):
    W1, b1, W2, b2, W3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    x, z1, h1, z2, h2 = acts
    gW3 = h2.T @ gy
    gb3 = gy.sum(axis=0)
    gh2 = gy @ W3.T
    gz2 = gh2 * (z2 > 0)
    gW2 = h1.T @ gz2
    gb2 = gz2.sum(axis=0)
    gh1 = gz2 @ W2.T
    gz1 = gh1 * (z1 > 0)
    gW1 = x.T @ gz1
    gb1 = gz1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3]


def loss(params, x, target) -> float:
    y, _ = forward(params, x)
    return loss_and_grad_out(y, target)[0]


def grads(params, x, target):
    y, acts = forward(params, x)
    l, gy = loss_and_grad_out(y, target)
    return l, backward(params, acts, gy)


def adam_step(master, grads_, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2015) with bias correction; returns new (master, m, v)."""
    out_p, out_m, out_v = [], [], []
    for p, g, mm, vv in zip(master, grads_, m, v):
        mm = b1 * mm + (1 - b1) * g
        vv = b2 * vv + (1 - b2) * g * g
        mh = mm / (1 - b1 ** step)
        vh = vv / (1 - b2 ** step)
        out_p.append(p - lr * mh / (np.sqrt(vh) + eps))
        out_m.append(mm)
        out_v.append(vv)
    return out_p, out_m, out_v

"""CPU oracle of the cardinality model (TEST INFRASTRUCTURE ONLY; the product path never
imports it). FP64 numpy forward and backward of the 3-layer MLP 32 -> 128 -> 128 -> 1 with
ReLU and a mean-squared-error loss, in two forms:

  exact      - no rounding anywhere (pinned against central finite differences);
  quantised  - the same network with every matmul input rounded to BF16 (round to nearest,
               ties to even) at the points where the GPU kernels round: the inputs, W1, W2,
               the hidden activations and the two back-propagated activation gradients.
               This is what the GPU result is compared with.

Parameters are one flat FP64 vector in the order W1[128][32] b1[128] W2[128][128] b2[128]
w3[128] b3 (the library's layout). The model is not from the paper; it is the learned
planner's cardinality estimator.
"""
from __future__ import annotations

import numpy as np

IN, H = 32, 128
SIZES = [H * IN, H, H * H, H, H, 1]


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = [], 0
    for s in SIZES:
        out.append(p[o:o + s])
        o += s
    W1, b1, W2, b2, w3, b3 = out
    return W1.reshape(H, IN), b1, W2.reshape(H, H), b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, np.atleast_1d(b3)]).astype(np.float64)


def bf16(x):
    """Round to the nearest BF16 value (ties to even) through FP32, returned as FP64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_backward(p, X, t=None, quantised=True):
    """Predictions, and with targets the MSE loss and its gradient (flat, parameter order)."""
    q = bf16 if quantised else (lambda v: np.asarray(v, dtype=np.float64))
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    Xq, W1q, W2q = q(X), q(W1), q(W2)
    Z1 = Xq @ W1q.T + b1
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2q.T + b2
    H2 = q(np.maximum(Z2, 0.0))
    y = H2 @ w3 + b3[0]
    if t is None:
        return y, None, None
    n = len(y)
    e = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / n
    dw3 = H2.T @ dy
    db3 = np.array([dy.sum()])
    dH2 = q(np.where(Z2 > 0, dy[:, None] * w3[None, :], 0.0))
    db2 = dH2.sum(axis=0)
    dW2 = dH2.T @ H1
    dA1 = dH2 @ W2q
    dH1 = q(np.where(Z1 > 0, dA1, 0.0))
    db1 = dH1.sum(axis=0)
    dW1 = dH1.T @ Xq
    return y, loss, pack(dW1, db1, dW2, db2, dw3, db3)


def init(seed: int):
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (H, IN)) * np.sqrt(6.0 / IN)
    W2 = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H)
    w3 = rng.uniform(-1, 1, H) * np.sqrt(3.0 / H)
    return pack(W1, rng.normal(0, 0.1, H), W2, rng.normal(0, 0.1, H), w3, np.array([0.2]))

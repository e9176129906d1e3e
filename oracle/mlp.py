"""CPU reference of the rank predictor (TEST INFRASTRUCTURE, FP64 numpy).

The network of the GPU path -- 6 -> 64 -> 64 -> 1 with ReLU, weights rounded
to BF16 -- evaluated and differentiated in FP64 with plain numpy, to check the
library's forward and backward kernels.  The parameter layout is the flat
4673-entry vector W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 6, 64
NPARAM = NH * NIN + NH + NH * NH + NH + NH + 1


def bf16_round(p: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even); returns FP64."""
    b = np.asarray(p, np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p: np.ndarray):
    o = 0
    W1 = p[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    w3 = p[o:o + NH]; o += NH
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p: np.ndarray, X: np.ndarray, round_bf16: bool = True) -> np.ndarray:
    q = bf16_round(p) if round_bf16 else np.asarray(p, np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(q)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss_grad(p: np.ndarray, X: np.ndarray, y: np.ndarray, round_bf16: bool = True):
    """Mean squared error and its gradient with respect to the (rounded)
    parameters, by back-propagation written out layer by layer."""
    q = bf16_round(p) if round_bf16 else np.asarray(p, np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(q)
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    out = h2 @ w3 + b3
    r = out - np.asarray(y, np.float64)
    loss = np.mean(r * r)
    dout = 2.0 * r / n
    gw3 = h2.T @ dout
    gb3 = dout.sum()
    d2 = np.outer(dout, w3) * (a2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g

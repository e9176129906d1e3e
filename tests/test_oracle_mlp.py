"""Pins of the predictor's CPU reference: finite differences for the
backward pass, the definition of bfloat16 rounding."""
import numpy as np

import hmat_synth as hs
from oracle import mlp


def test_bf16_rounding_definition():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3.0e38, 1e-40], np.float32)
    r = mlp.bf16_round(x)
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie -> even (1.0),
    # 1 + 3 * 2^-8 is a tie -> even (1 + 2^-6)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7 and r[3] == 1.0 + 2 ** -6
    assert r[4] == -2.5
    assert abs(r[5] - 3.0e38) / 3.0e38 < 2 ** -8
    # below the normal range bfloat16 steps by 2^-133; 1e-40 is nearest to one step
    assert r[6] == 2.0 ** -133


def test_backward_matches_finite_differences():
    p = hs.normal(1, mlp.NPARAM) * 0.3
    X = hs.normal(2, 40 * 6).reshape(40, 6)
    y = hs.normal(3, 40)
    loss, g = mlp.loss_grad(p, X, y, round_bf16=False)
    idx = np.concatenate([np.arange(0, 384, 37), np.arange(384, 448, 9), np.arange(448, 4544, 301),
                          np.arange(4544, 4673, 11), [4672]])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        lp, _ = mlp.loss_grad(p + e, X, y, round_bf16=False)
        lm, _ = mlp.loss_grad(p - e, X, y, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_forward_is_the_network():
    p = hs.normal(4, mlp.NPARAM) * 0.2
    X = hs.normal(5, 6).reshape(1, 6)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(mlp.bf16_round(p.astype(np.float32)))
    h = np.maximum(W1 @ X[0] + b1, 0)
    h = np.maximum(W2 @ h + b2, 0)
    assert np.isclose(mlp.forward(p.astype(np.float32), X)[0], w3 @ h + b3)

"""CPU pins of the FP64 order-model reference: backprop against central
differences, and the BF16 rounding helper against exact cases."""
import numpy as np

import mlp_ref


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.3, mlp_ref.NPARAMS)
    X = rng.normal(0, 1, (40, 8))
    y = rng.integers(0, 6, 40)
    _, g = mlp_ref.loss_and_grad(p, X, y)
    idx = rng.choice(mlp_ref.NPARAMS, 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        num = (mlp_ref.loss_and_grad(p + e, X, y)[0] - mlp_ref.loss_and_grad(p - e, X, y)[0]) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num))


def test_bf16_round():
    assert mlp_ref.bf16_round(1.0) == 1.0
    assert mlp_ref.bf16_round(1.0 + 2 ** -9) == 1.0          # ties to even
    assert mlp_ref.bf16_round(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp_ref.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)

"""The FP64 twin of the warm-start network: analytic gradient pinned against
central finite differences (CPU only)."""
import numpy as np

from oracle import mlp


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.2, size=mlp.n_params())
    X = rng.normal(size=(7, mlp.F_IN))
    t = rng.normal(size=7)
    L, g = mlp.loss_and_grad(theta, X, t)
    assert abs(L - mlp.loss(theta, X, t)) < 1e-15 * max(1.0, L)
    idx = rng.choice(mlp.n_params(), size=60, replace=False)
    idx = np.concatenate([idx, [mlp.n_params() - 1, 0, 2048, 2048 + 128]])   # b4, W1, b1, W2 starts
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (mlp.loss(tp, X, t) - mlp.loss(tm, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_bf16_rounding():
    """bfloat16 keeps 8 significant bits; halfway cases round to even."""
    x = np.array([1.00390625, 1.001953125, 1.01171875, -3.14159, 0.0, 1.0078125])
    r = mlp.bf16(x)
    assert r[0] == 1.0            # 1 + 2^-8: halfway between 1 and 1 + 2^-7, even is 1
    assert r[1] == 1.0            # below halfway
    assert r[2] == 1.015625       # 1 + 3*2^-8: halfway, even neighbour is 1 + 2^-6
    assert r[3] == -3.140625
    assert r[4] == 0.0
    assert r[5] == 1.0078125      # representable

"""The FP64 twin of the warm-start network: forward pass pinned by closed-form
special cases, analytic gradient pinned against
central finite differences (CPU only)."""
import math

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


def _zero():
    return [np.zeros(s) for s in mlp.SHAPES]


def _silu(z):
    return z / (1.0 + math.exp(-z))


def test_forward_output_layer_closed_form():
    """All hidden weights zero: A3 = silu(b3) on every row, so out = w4 . silu(b3) + b4.
    With b3 = (ln 3, 0, -ln 3) and w4 = (1, 1, 1): silu(ln 3) = 3/4 ln 3 and
    silu(-ln 3) = -1/4 ln 3, so out = 1/2 ln 3 + b4; and the loss against
    t = out + 2 is 4."""
    P = _zero()
    P[5][:3] = [math.log(3.0), 0.0, -math.log(3.0)]
    P[6][:3] = 1.0
    P[7][0] = 0.37
    X = np.random.default_rng(1).normal(size=(5, mlp.F_IN))
    out, _ = mlp.forward(mlp.pack(P), X)
    assert np.allclose(out, 0.5 * math.log(3.0) + 0.37, rtol=0, atol=1e-15)
    assert abs(mlp.loss(mlp.pack(P), X, out + 2.0) - 4.0) < 1e-14


def test_forward_single_path_follows_the_packing():
    """One nonzero weight per layer on the path input 5 -> unit 7 -> unit 3 ->
    unit 11 -> output (row-major W1[16x128], W2, W3[128x128]): the output is
    silu(silu(silu(x_5))), computed here with scalar math.  A transposed
    matrix or a misplaced block of the packing routes the path through a zero."""
    P = _zero()
    P[0][5, 7] = 1.0
    P[2][7, 3] = 1.0
    P[4][3, 11] = 1.0
    P[6][11] = 1.0
    X = np.zeros((3, mlp.F_IN))
    X[:, 5] = [math.log(3.0), -0.7, 2.5]
    out, _ = mlp.forward(mlp.pack(P), X)
    ref = [_silu(_silu(_silu(z))) for z in X[:, 5]]
    assert np.allclose(out, ref, rtol=1e-15, atol=1e-15)
    # the same path driven by the biases b1 (unit 7) and b2 (unit 3) instead
    for layer, unit, down in ((1, 7, None), (3, 3, 0)):
        Q = [p.copy() for p in P]
        Q[0][:] = 0.0
        if down is not None:
            Q[2][:] = 0.0
        Q[layer][unit] = 1.25
        out2, _ = mlp.forward(mlp.pack(Q), np.zeros((1, mlp.F_IN)))
        expect = _silu(_silu(_silu(1.25))) if layer == 1 else _silu(_silu(1.25))
        assert abs(out2[0] - expect) < 1e-15, (layer, out2[0], expect)

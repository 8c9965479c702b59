"""FP64 twin of the warm-start network (test infrastructure).

Network: X[rows, 16] -> Z1 = X W1 + b1 -> A1 = silu(Z1) -> Z2 = A1 W2 + b2 -> A2 =
silu(Z2) -> Z3 = A2 W3 + b3 -> A3 = silu(Z3) -> out = A3 w4 + b4, loss =
mean((out - t)^2), silu(z) = z / (1 + exp(-z)).  Parameters are packed in the
order W1 (16x128, row-major), b1, W2 (128x128), b2, W3 (128x128), b3, w4 (128), b4.

``bf16=True`` rounds the network inputs, the weights of the matrix products and
the stored activations to bfloat16 (round to nearest even), as the GPU kernels
store them, while every sum stays in FP64; the remaining difference to the GPU
is then the FP32 accumulation order only.

The backward pass is the chain rule written out; tests pin it against central
finite differences of ``loss``.  The paper has no network, so nothing in it pins
this twin (parity unpinned by the paper): its forward pass is pinned by
closed-form special cases (an output layer alone, single paths through the
packed weights and biases), its gradient by finite differences.
"""
from __future__ import annotations

import numpy as np

F_IN, HID = 16, 128
SHAPES = [(F_IN, HID), (HID,), (HID, HID), (HID,), (HID, HID), (HID,), (HID,), (1,)]


def n_params() -> int:
    return int(sum(np.prod(s) for s in SHAPES))


def unpack(theta):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def bf16(a):
    """Round to bfloat16 (nearest even) and return as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X, bf16_mode=False):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(theta)
    r = bf16 if bf16_mode else (lambda a: np.asarray(a, dtype=np.float64))
    X = r(X)
    Z1 = X @ r(W1) + b1
    A1 = r(_silu(Z1))
    Z2 = A1 @ r(W2) + b2
    A2 = r(_silu(Z2))
    Z3 = A2 @ r(W3) + b3
    A3 = r(_silu(Z3))
    out = A3 @ r(w4) + b4[0]
    return out, (X, Z1, A1, Z2, A2, Z3, A3)


def loss(theta, X, t, bf16_mode=False):
    out, _ = forward(theta, X, bf16_mode)
    return float(np.mean((out - np.asarray(t, dtype=np.float64)) ** 2))


def loss_and_grad(theta, X, t, bf16_mode=False):
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(theta)
    r = bf16 if bf16_mode else (lambda a: np.asarray(a, dtype=np.float64))
    out, (Xr, Z1, A1, Z2, A2, Z3, A3) = forward(theta, X, bf16_mode)
    t = np.asarray(t, dtype=np.float64)
    rows = len(t)
    L = float(np.mean((out - t) ** 2))
    dout = 2.0 * (out - t) / rows
    gw4 = A3.T @ dout
    gb4 = np.array([dout.sum()])
    dZ3 = np.outer(dout, r(w4)) * _dsilu(Z3)
    gW3 = A2.T @ dZ3
    gb3 = dZ3.sum(axis=0)
    dZ2 = (dZ3 @ r(W3).T) * _dsilu(Z2)
    gW2 = A1.T @ dZ2
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ r(W2).T) * _dsilu(Z1)
    gW1 = Xr.T @ dZ1
    gb1 = dZ1.sum(axis=0)
    return L, pack([gW1, gb1, gW2, gb2, gW3, gb3, gw4, gb4])

"""Training pipeline of the learned warm start (calls the C ABI only).

For each training problem the solver computes the ground state (FP64), the
library fits the per-orbit weights w* of the product vector exp(sum_{i in s}
w_i) to it, and the network is trained to map per-orbit features to w*.
"""
from __future__ import annotations

import numpy as np

from . import pairdiag as pd


def training_set(problems, tol: float = 1e-10):
    """problems: iterable of (omega, n_pairs, e, G).  Returns (X, targets)."""
    import torch
    X_rows, T_rows = [], []
    for omega, n, e, G in problems:
        with pd.Solver(omega, n, e, G, precision=pd.PD_PREC_FP64) as s:
            v = torch.empty(s.dim, dtype=torch.float64, device="cuda")
            pd.pairdiag_ground_state_dev(s.h, tol, v)
            w = pd.pairdiag_product_fit(s.h, v, omega)
        X_rows.append(pd.pairdiag_mlp_features(omega, n, e, G))
        T_rows.append(w.astype(np.float32))
    return np.concatenate(X_rows), np.concatenate(T_rows)


class WarmStart:
    """A trained network; ``attach(handle)`` makes PD_START_MLP use it."""

    def __init__(self, seed: int = 0, params=None):
        self.m = pd.pairdiag_mlp_create(seed)
        if params is not None:
            pd.pairdiag_mlp_set_params(self.m, params)

    def train(self, X, T, steps: int = 3000, lr: float = 2e-3):
        return pd.pairdiag_mlp_train(self.m, X, T, steps, lr)

    def predict(self, omega, n, e, G):
        return pd.pairdiag_mlp_forward(self.m, pd.pairdiag_mlp_features(omega, n, e, G))

    def params(self):
        return pd.pairdiag_mlp_get_params(self.m)

    def attach(self, h):
        pd.pairdiag_set_mlp(h, self.m)

    def close(self):
        if self.m is not None:
            pd.pairdiag_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

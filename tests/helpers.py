"""Shared helpers of the GPU parity tests (tolerances derived from the arithmetic)."""
import math

import numpy as np

import oracle

EPS64 = np.finfo(np.float64).eps
EPS32 = float(np.finfo(np.float32).eps)


def abs_row_scale(omega, n, e, G, x, rows=None, basis=None):
    """(|H| |x|) per row: the sum of absolute values of every term of a row of
    H x, computed by the oracle on |G| and a diagonal of sum_p |2 e_p + G_pp|."""
    G = np.asarray(G, dtype=np.float64)
    d = 2.0 * np.asarray(e) + np.diag(G)
    Gabs = np.abs(G)
    e_abs = (np.abs(d) - np.diag(Gabs)) / 2.0
    if rows is None:
        return oracle.hx(omega, n, e_abs, Gabs, np.abs(x), basis)
    return oracle.hx_rows(omega, n, e_abs, Gabs, np.abs(x), rows, basis)


def hx_bound(omega, n, scale, eps):
    """Worst-case rounding bound for a reordered sum of nnz_row + 1 products
    (plus the rounding of the inputs): 4 (N(Omega-N) + 2) eps |H||x|."""
    terms = n * (omega - n) + 2
    return 4.0 * terms * eps * scale


def comb(omega, n):
    return math.comb(omega, n)


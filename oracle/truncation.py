"""The truncated model space of Sec. 3.5 (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; it shares no code with the CUDA path.

When C(Omega, N) exceeds Dimension_Limit, the paper keeps the basis states
with the lowest diagonal elements: it histograms every diagonal element into
10^8 equal bins between the smallest and the largest, counts bins from the
bottom until about Dimension_Limit states lie below the cutoff, and drops every
state above it.  The kept states stay in the basis order (ascending integer
order), and a scattered state is located by binary search; a hop to a dropped
state contributes nothing, so the truncated operator is the principal
submatrix of H on the kept states.

Readings of the passage (it says "approximately equal"):
  * a diagonal element d falls in bin floor((d - min) / (max - min) * bins),
    computed in FP64, with the maximum put in the last bin;
  * the cutoff bin is the lowest bin at which the running count reaches
    Dimension_Limit, and every state in a bin up to and including it is kept,
    so at least Dimension_Limit states are kept (more when the cutoff bin holds
    several);
  * no truncation when C(Omega, N) <= Dimension_Limit, or when every diagonal
    element is equal.

Pinned in tests/test_oracle_truncation.py (interlacing, nesting, the sorted
cutoff, the dense principal submatrix, the paper's remark that weak pairing
tolerates more truncation).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import basis as _basis, diag as _diag, lib, _f64, _p

DEFAULT_BINS = 10 ** 8


def diagonals(omega: int, n: int, e, G, b: np.ndarray | None = None) -> np.ndarray:
    """Eq. (diagonal) for every basis state, in basis order."""
    if b is None:
        b = _basis(omega, n)
    return np.array([_diag(int(s), e, G) for s in b])


def cutoff_bin(d: np.ndarray, limit: int, bins: int = DEFAULT_BINS):
    """(bin index of every element, cutoff bin) of the histogram of Sec. 3.5."""
    lo, hi = float(d.min()), float(d.max())
    if hi == lo:
        return np.zeros(len(d), dtype=np.int64), 0
    idx = np.floor((d - lo) / (hi - lo) * bins).astype(np.int64)
    idx = np.minimum(idx, bins - 1)
    k = min(limit, len(d))
    cut = int(np.partition(idx, k - 1)[k - 1])       # lowest bin whose running count reaches k
    return idx, cut


def truncate(omega: int, n: int, e, G, limit: int, bins: int = DEFAULT_BINS) -> dict:
    """Kept states (ascending), their count, the cutoff bin and the full dimension."""
    if limit < 1:
        raise ValueError("limit must be >= 1")
    b = _basis(omega, n)
    if len(b) <= limit:
        return dict(kept=b, dim=len(b), full_dim=len(b), cut_bin=None, truncated=False)
    d = diagonals(omega, n, e, G, b)
    idx, cut = cutoff_bin(d, limit, bins)
    kept = b[idx <= cut]
    return dict(kept=kept, dim=len(kept), full_dim=len(b), cut_bin=cut, truncated=len(kept) < len(b))


def hx_sub(omega: int, e, G, kept: np.ndarray, x) -> np.ndarray:
    """H x on the kept states (the principal submatrix), binary search per hop."""
    e = _f64(e); G = _f64(G); x = _f64(x)
    kept = np.ascontiguousarray(kept, dtype=np.uint64)
    y = np.empty(len(kept))
    lib().orc_hx_sub(omega, _p(e), _p(G), _p(kept), len(kept), _p(x), _p(y))
    return y


def sub_matrix(omega: int, e, G, kept: np.ndarray) -> np.ndarray:
    """The truncated matrix, column by column from hx_sub (small spaces only)."""
    m = len(kept)
    M = np.empty((m, m))
    x = np.zeros(m)
    for j in range(m):
        x[:] = 0.0; x[j] = 1.0
        M[:, j] = hx_sub(omega, e, G, kept, x)
    return M


def ground_energy(omega: int, n: int, e, G, limit: int, bins: int = DEFAULT_BINS) -> float:
    """Lowest eigenvalue of H on the truncated space (dense, small spaces only)."""
    t = truncate(omega, n, e, G, limit, bins)
    return float(np.linalg.eigvalsh(sub_matrix(omega, e, G, t["kept"]))[0])

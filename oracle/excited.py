"""The lowest few eigenpairs of the pairing Hamiltonian (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; it shares no code with the CUDA path.

Sec. 3.4 chooses Lanczos because only the first few states of the pairing
Hamiltonian are wanted.  Their plain definition is the k lowest eigenvalues of
the dim x dim matrix of Eq. 2 with orthonormal eigenvectors; this module
computes exactly that for small dimensions: the dense matrix assembled column by
column from the oracle's H*x by explicit scattering (Sec. 3.3), then a dense
symmetric eigensolver (one library step).

Pinned in tests/test_oracle_excited.py: the quasispin spectrum of a degenerate
level with its multiplicities, the trace of the matrix, the oracle's own cyclic
Jacobi, the seniority-zero block of Eq. 1 built in the fermion Fock space, and
the restarted-Lanczos ground state.
"""
from __future__ import annotations

import numpy as np

from . import dense_matrix


def lowest_k(omega: int, n: int, e, G, k: int):
    """(energies [k], vectors [dim, k]) of the k lowest eigenpairs, ascending;
    vectors orthonormal, in the basis order of Sec. 3.1."""
    M = dense_matrix(omega, n, e, G)
    if not 1 <= k <= M.shape[0]:
        raise ValueError("k outside 1..dim")
    w, V = np.linalg.eigh(M)
    return w[:k].copy(), V[:, :k].copy()

"""Odd-mass ground state in the blocking approximation (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; it shares no code with the CUDA path.

Eq. 3: with one unpaired particle in orbit b, the Pauli principle keeps every
pair out of b.  The seniority-one subspace in which b is blocked is therefore
the seniority-zero space of the N pairs on the remaining Omega-1 orbits, and
H_b acts there as the constant e_b (the odd particle's single-particle energy)
plus the Hamiltonian of Eq. 2 with its sums restricted to orbits other than b.
The paper's Block argument (Sec. 4.2) picks the subspaces: Block = 0 solves
every b and returns the lowest ground state, Block = b solves b alone; here
``block=None`` and a 0-based orbit index play those roles.  The occupation
output N_Occup (Sec. 4.3) is 2<S+_i S-_i> for the paired orbits and 1 for the
blocked one.

Each subspace is solved by the oracle's own restarted Lanczos (Algorithm 2).
Pinned in tests/test_oracle_odd.py against the Hamiltonian of Eq. 1 built by
brute force in the full fermion Fock space, the seniority formula of a
degenerate level, and Richardson's equations on the unblocked orbits.
"""
from __future__ import annotations

import numpy as np

from . import basis as _basis, lanczos_ground


def reduced_problem(e, G, b: int):
    """(e, G) with orbit b removed; the other orbits keep their order."""
    e = np.asarray(e, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    keep = np.array([i for i in range(len(e)) if i != b], dtype=np.int64)
    return e[keep].copy(), G[np.ix_(keep, keep)].copy(), keep


def occupations(omega: int, n: int, v) -> np.ndarray:
    """N_Occup (Sec. 4.3) of a normalised seniority-zero vector: 2 sum_s v_s^2 n_i(s),
    n_i(s) = 1 when orbit i holds a pair in basis state s."""
    v = np.asarray(v, dtype=np.float64)
    b = _basis(omega, n)
    occ = np.zeros(omega)
    for i in range(omega):
        bit = ((b >> np.uint64(i)) & np.uint64(1)).astype(bool)
        occ[i] = 2.0 * float(np.sum(v[bit] ** 2))
    return occ


def blocked_ground(omega: int, n: int, e, G, block: int | None = None, tol: float = 1e-12,
                   window: int = 50, max_restarts: int = 500) -> dict:
    """Lowest eigenpair of H_b (Eq. 3) for 2n+1 particles on omega orbits.

    block None: every b in 0..omega-1, returning the lowest (the paper's Block = 0);
    otherwise that orbit only.  Returns e0, block, energies (omega entries, NaN for
    subspaces not solved), occ (omega), vec (the pair vector on the omega-1
    unblocked orbits, in their basis order) and converged."""
    if omega < 2 or not 0 <= n <= omega - 1:
        raise ValueError("need omega >= 2 and 0 <= n <= omega - 1")
    blocks = range(omega) if block is None else [int(block)]
    energies = np.full(omega, np.nan)
    best = None
    converged = True
    for b in blocks:
        if not 0 <= b < omega:
            raise ValueError("block outside 0..omega-1")
        er, Gr, keep = reduced_problem(e, G, b)
        r = lanczos_ground(omega - 1, n, er, Gr, window=window, tol=tol, max_restarts=max_restarts)
        converged = converged and r["converged"]
        energies[b] = float(np.asarray(e, dtype=np.float64)[b]) + r["e0"]
        if best is None or energies[b] < energies[best[0]]:
            best = (b, r, keep)
    b, r, keep = best
    vec = r["vec"] / np.linalg.norm(r["vec"])
    occ = np.zeros(omega)
    occ[keep] = occupations(omega - 1, n, vec)
    occ[b] = 1.0
    return dict(e0=float(energies[b]), block=b, energies=energies, occ=occ, vec=vec, converged=converged)

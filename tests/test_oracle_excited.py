"""Pins of the excited-state oracle (the lowest few eigenpairs, Sec. 3.4; CPU only)."""
import math

import numpy as np
import pytest

import oracle
from oracle import excited
from test_oracle_odd import fock_hamiltonian, _pattern, _random_problem


def quasispin_levels(omega, n, eps, g):
    """Spectrum of a degenerate level (e_i = eps, V_ij = g) in the pair space.

    The pair operators of the Omega orbits are Omega spin-1/2 raising operators,
    so sum_ij P_i^+ P_j = S+ S- = S^2 - S_z^2 + S_z with S_z = n - Omega/2.  Total
    quasispin S = Omega/2 - t (t = 0..min(n, Omega-n)) occurs C(Omega,t) -
    C(Omega,t-1) times at fixed S_z, which gives
        E_t = 2 eps n + g [n (Omega - n + 1) - t (Omega + 1 - t)]."""
    out = []
    for t in range(min(n, omega - n) + 1):
        mult = math.comb(omega, t) - (math.comb(omega, t - 1) if t else 0)
        out += [2 * eps * n + g * (n * (omega - n + 1) - t * (omega + 1 - t))] * mult
    return np.array(sorted(out))


@pytest.mark.parametrize("omega,n", [(8, 4), (10, 3), (9, 9), (7, 0)])
def test_degenerate_level_full_spectrum(omega, n):
    eps, g = 0.6, -0.35
    dim = math.comb(omega, n)
    w, V = excited.lowest_k(omega, n, np.full(omega, eps), np.full((omega, omega), g), dim)
    ref = quasispin_levels(omega, n, eps, g)
    assert len(ref) == dim
    assert np.allclose(w, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
    assert np.allclose(V.T @ V, np.eye(dim), atol=1e-12)


def test_trace_and_jacobi_agree():
    omega, n, k = 8, 3, 56
    e, G = _random_problem(omega, 41)
    w, V = excited.lowest_k(omega, n, e, G, k)
    d = 2 * e + np.diag(G)
    assert abs(w.sum() - math.comb(omega - 1, n - 1) * d.sum()) <= 1e-11 * np.abs(w).sum()
    wj, _ = oracle.jacobi(oracle.dense_matrix(omega, n, e, G))
    assert np.allclose(w, np.sort(wj), rtol=0, atol=1e-11)
    M = oracle.dense_matrix(omega, n, e, G)
    assert np.allclose(M @ V, V * w, atol=1e-11)


@pytest.mark.parametrize("omega,n,seed", [(5, 2, 51), (6, 3, 52)])
def test_spectrum_matches_eq1_seniority_zero_block(omega, n, seed):
    """Every eigenvalue of the paired Fock states of Eq. 1 (2n particles)."""
    e, G = _random_problem(omega, seed)
    states, H = fock_hamiltonian(e, G, 2 * n)
    sel = [k for k, s in enumerate(states) if all(x in (0, 2) for x in _pattern(s, omega))]
    ref = np.linalg.eigvalsh(H[np.ix_(sel, sel)])
    w, _ = excited.lowest_k(omega, n, e, G, len(sel))
    assert np.allclose(w, ref, rtol=0, atol=1e-11)


def test_lowest_is_the_lanczos_ground_state():
    omega, n = 10, 5
    e, G = _random_problem(omega, 61)
    w, V = excited.lowest_k(omega, n, e, G, 3)
    r = oracle.lanczos_ground(omega, n, e, G, tol=1e-13)
    assert abs(w[0] - r["e0"]) <= 1e-11 * abs(w[0])
    assert abs(abs(V[:, 0] @ r["vec"]) - 1.0) < 1e-10
    assert w[0] < w[1] <= w[2]

"""Pins of the excited-state oracle (the lowest few eigenpairs, Sec. 3.4; CPU only)."""
import math

import numpy as np
import pytest

import oracle
import pd_inputs
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


def _locked_lanczos(M, locked, start, tol=1e-12, m=20, cycles=200):
    """A plain model of restarted Lanczos on M projected against the locked
    vectors (full reorthogonalisation, restart from the lowest Ritz vector)."""
    q = start.copy()
    for _ in range(cycles):
        for l in locked:
            q -= l * (l @ q)
        q /= np.linalg.norm(q)
        Q, a, b = [q], [], []
        for i in range(m):
            p = M @ Q[i]
            for l in locked:
                p -= l * (l @ p)
            a.append(Q[i] @ p)
            p -= a[-1] * Q[i]
            if i:
                p -= b[-1] * Q[i - 1]
            for v in Q:
                p -= v * (v @ p)
            beta = np.linalg.norm(p)
            if i == m - 1 or beta < 1e-13 * max(abs(x) for x in a):
                break
            b.append(beta)
            Q.append(p / beta)
        T = np.diag(a) + np.diag(b[:len(a) - 1], 1) + np.diag(b[:len(a) - 1], -1)
        w, S = np.linalg.eigh(T)
        q = np.array(Q[:len(a)]).T @ S[:, 0]
        if np.linalg.norm(M @ q - w[0] * q) <= tol * abs(w[0]):
            break
    return w[0], q / np.linalg.norm(q)


def test_locking_needs_a_fresh_start_per_state():
    """The reading behind the lowest-states entry point.  On a degenerate level a
    start vector reused after projection has no component left in the rest of
    the eigenspace once one copy is locked, so the next solve skips the other
    copies; a fresh random start per state finds every copy, in order."""
    omega, n, eps, g, k = 10, 4, 0.5, -0.3, 6
    M = oracle.dense_matrix(omega, n, np.full(omega, eps), np.full((omega, omega), g))
    ref = quasispin_levels(omega, n, eps, g)[:k]
    found = {}
    for label, seeds in (("reused", [1] * k), ("fresh", list(range(1, k + 1)))):
        locked, energies = [], []
        for j in range(k):
            start = pd_inputs.splitmix_uniform(seeds[j], M.shape[0])
            ej, v = _locked_lanczos(M, locked, start)
            energies.append(ej)
            locked.append(v)
        found[label] = np.array(energies)
    assert np.allclose(found["fresh"], ref, rtol=0, atol=1e-10)
    assert not np.allclose(found["reused"], ref, rtol=0, atol=1e-6)
    assert found["reused"][2] > ref[2] + 1.0        # jumps to a higher level

"""Pins of the odd-mass (blocking) oracle, Eq. 3 (CPU only).

The strongest pin builds the Hamiltonian of Eq. 1 itself, by brute force, in
the full Fock space of 2*Omega fermion states (i and its time-reversed partner
ibar), with Jordan-Wigner signs; nothing there assumes pairs, blocking or the
diagonal of Eq. 2.  The other pins are the seniority formula of a degenerate
level and Richardson's equations on the unblocked orbits.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import odd, richardson


# ---- Eq. 1 in the fermion Fock space -------------------------------------------
# mode 2i is state i, mode 2i+1 its time-reversed partner ibar

def _apply(ops, state):
    """Apply a product of ladder operators, rightmost first, to a Fock state
    (bitmask).  ops: sequence of (mode, create).  Returns (sign, state) or None."""
    sign = 1
    for mode, create in reversed(ops):
        occupied = (state >> mode) & 1
        if occupied == create:
            return None
        if bin(state & ((1 << mode) - 1)).count("1") % 2:
            sign = -sign
        state ^= 1 << mode
    return sign, state


def fock_hamiltonian(e, V, n_particles):
    """Matrix of Eq. 1, H = sum_i e_i a+_i a_i + sum_{ii'} V_ii' a+_i a+_ibar a_i'bar a_i',
    on every Fock state of n_particles fermions in 2*Omega modes (the one-body sum
    runs over both members of each pair of states)."""
    omega = len(e)
    states = [sum(1 << m for m in c) for c in itertools.combinations(range(2 * omega), n_particles)]
    index = {s: k for k, s in enumerate(states)}
    H = np.zeros((len(states), len(states)))
    terms = []
    for i in range(omega):
        for m in (2 * i, 2 * i + 1):
            terms.append((e[i], [(m, 1), (m, 0)]))
    for i in range(omega):
        for j in range(omega):
            terms.append((V[i][j], [(2 * i, 1), (2 * i + 1, 1), (2 * j + 1, 0), (2 * j, 0)]))
    for col, s in enumerate(states):
        for coef, ops in terms:
            r = _apply(ops, s)
            if r is not None:
                H[index[r[1]], col] += coef * r[0]
    return states, H


def _pattern(s, omega):
    """Per orbit: 0 empty, 2 paired, ('i' or 'ibar') singly occupied."""
    out = []
    for i in range(omega):
        a, b = (s >> (2 * i)) & 1, (s >> (2 * i + 1)) & 1
        out.append(2 if a and b else 0 if not (a or b) else ("i" if a else "ibar"))
    return out


def _random_problem(omega, seed):
    rng = np.random.default_rng(seed)
    e = np.sort(rng.uniform(-2.0, 2.0, omega))
    g = rng.uniform(0.3, 0.7, omega)
    eta = rng.normal(0.0, 0.1, (omega, omega))
    G = -np.outer(g, g) + (eta + eta.T) / 2.0
    return e, G


@pytest.mark.parametrize("omega,n,seed", [(4, 1, 11), (5, 2, 12), (6, 2, 13)])
def test_blocked_subspaces_match_eq1_in_fock_space(omega, n, seed):
    """For each b, the Fock states with orbit b singly occupied (by state b) and every
    other orbit empty or paired are closed under Eq. 1 (Pauli blocking), and the
    lowest eigenvalue there is E_b of the oracle; the occupations match too."""
    e, G = _random_problem(omega, seed)
    states, H = fock_hamiltonian(e, G, 2 * n + 1)
    assert np.array_equal(H, H.T)
    pats = [_pattern(s, omega) for s in states]
    r_all = odd.blocked_ground(omega, n, e, G)
    for b in range(omega):
        sel = [k for k, p in enumerate(pats)
               if p[b] == "i" and all(x in (0, 2) for i, x in enumerate(p) if i != b)]
        assert len(sel) == oracle.binom(omega - 1, n)
        rest = [k for k in range(len(states)) if k not in set(sel)]
        assert np.all(H[np.ix_(rest, sel)] == 0.0)          # nothing leaves the subspace
        w, U = np.linalg.eigh(H[np.ix_(sel, sel)])
        r = odd.blocked_ground(omega, n, e, G, block=b)
        assert abs(r["e0"] - w[0]) <= 1e-11 * max(1.0, abs(w[0]))
        assert abs(r_all["energies"][b] - w[0]) <= 1e-11 * max(1.0, abs(w[0]))
        u = U[:, 0]
        occ = np.zeros(omega)
        for amp, k in zip(u, sel):
            s = states[k]
            for i in range(omega):
                occ[i] += amp * amp * (((s >> (2 * i)) & 1) + ((s >> (2 * i + 1)) & 1))
        if w[1] - w[0] > 1e-6:
            assert np.allclose(r["occ"], occ, atol=1e-9)
    assert r_all["block"] == int(np.nanargmin(r_all["energies"]))


@pytest.mark.parametrize("omega,n,seed", [(5, 2, 21), (6, 3, 22)])
def test_even_seniority_zero_block_matches_eq2(omega, n, seed):
    """The paired Fock states of 2n particles carry the lowest seniority-zero
    eigenvalue of Eq. 2 with diagonal 2 e_i + V_ii: the even-mass oracle."""
    e, G = _random_problem(omega, seed)
    states, H = fock_hamiltonian(e, G, 2 * n)
    sel = [k for k, s in enumerate(states) if all(x in (0, 2) for x in _pattern(s, omega))]
    assert len(sel) == oracle.binom(omega, n)
    w = np.linalg.eigvalsh(H[np.ix_(sel, sel)])
    r = oracle.lanczos_ground(omega, n, e, G, tol=1e-13)
    assert abs(r["e0"] - w[0]) <= 1e-11 * max(1.0, abs(w[0]))


@pytest.mark.parametrize("omega,n", [(8, 3), (10, 4), (9, 0), (7, 6)])
def test_degenerate_level_seniority_formula(omega, n):
    """A degenerate level (e_i = eps, V_ij = g) with one unpaired particle has the
    seniority-one energy eps (2n+1) + g n (Omega - n) for every blocked orbit."""
    eps, g = 0.7, -0.3
    e = np.full(omega, eps)
    G = np.full((omega, omega), g)
    r = odd.blocked_ground(omega, n, e, G)
    exact = eps * (2 * n + 1) + g * n * (omega - n)
    assert np.allclose(r["energies"], exact, rtol=0, atol=1e-11 * max(1.0, abs(exact)))
    assert abs(r["e0"] - exact) <= 1e-11 * max(1.0, abs(exact))
    assert r["occ"][r["block"]] == 1.0
    assert abs(r["occ"].sum() - (2 * n + 1)) <= 1e-10


def test_constant_g_blocked_orbits_match_richardson():
    """Constant G: E_b = e_b + (Richardson energy of the other orbits), for every b."""
    omega, n, g = 12, 5, -0.4
    e = np.arange(1.0, omega + 1.0) + 0.013 * np.sin(np.arange(omega))
    G = np.full((omega, omega), g)
    r = odd.blocked_ground(omega, n, e, G)
    for b in range(omega):
        er = np.delete(e, b)
        ref = e[b] + richardson.ground_energy(er, g, n)
        assert abs(r["energies"][b] - ref) <= 1e-10 * abs(ref), b
    assert r["block"] == int(np.argmin(r["energies"]))


def test_occupation_sum_rule_and_block_choice():
    omega, n = 10, 4
    e, G = _random_problem(omega, 31)
    r = odd.blocked_ground(omega, n, e, G)
    assert r["occ"][r["block"]] == 1.0
    assert abs(r["occ"].sum() - (2 * n + 1)) <= 1e-10
    assert np.all(r["occ"] >= -1e-12) and np.all(r["occ"] <= 2.0 + 1e-12)
    assert r["e0"] == np.min(r["energies"])
    one = odd.blocked_ground(omega, n, e, G, block=r["block"])
    assert abs(one["e0"] - r["e0"]) <= 1e-12 * abs(r["e0"])
    assert np.isnan(one["energies"]).sum() == omega - 1


# ---- planted mistakes: each must break a pin above -------------------------------

ODD_MUTATIONS = {
    "blocked_pair_energy": ("energies[b] = float(np.asarray(e, dtype=np.float64)[b]) + r[\"e0\"]",
                            "energies[b] = 2.0 * float(np.asarray(e, dtype=np.float64)[b]) + r[\"e0\"]"),
    "blocked_orbit_keeps_its_interaction": ("G[np.ix_(keep, keep)].copy()",
                                            "G[:len(e) - 1, :len(e) - 1].copy()"),
    "blocked_occupancy_two": ("occ[b] = 1.0", "occ[b] = 2.0"),
    "highest_subspace": ("energies[b] < energies[best[0]]", "energies[b] > energies[best[0]]"),
}


def _mutant(old, new):
    import types
    from pathlib import Path
    src = Path(odd.__file__).read_text()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle._odd_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), "odd_mutant.py", "exec"), mod.__dict__)
    return mod


def _odd_pins_hold(mod) -> bool:
    omega, n = 5, 2
    e, G = _random_problem(omega, 12)
    states, H = fock_hamiltonian(e, G, 2 * n + 1)
    pats = [_pattern(s, omega) for s in states]
    r_all = mod.blocked_ground(omega, n, e, G)
    lows = []
    for b in range(omega):
        sel = [k for k, p in enumerate(pats)
               if p[b] == "i" and all(x in (0, 2) for i, x in enumerate(p) if i != b)]
        lows.append(np.linalg.eigvalsh(H[np.ix_(sel, sel)])[0])
    if not np.allclose(r_all["energies"], lows, rtol=0, atol=1e-10):
        return False
    if abs(r_all["e0"] - min(lows)) > 1e-10:
        return False
    return r_all["occ"][r_all["block"]] == 1.0 and abs(r_all["occ"].sum() - (2 * n + 1)) < 1e-10


def test_unmutated_odd_oracle_passes_the_pin_set():
    assert _odd_pins_hold(odd)


@pytest.mark.parametrize("name", sorted(ODD_MUTATIONS))
def test_planted_odd_mistake_is_caught(name):
    assert not _odd_pins_hold(_mutant(*ODD_MUTATIONS[name]))

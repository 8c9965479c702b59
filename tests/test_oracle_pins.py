"""Pins of the CPU oracle against the paper's printed values, closed forms,
invariants and brute force (no GPU needed)."""
import itertools
import math

import numpy as np
import pytest

import oracle
import pd_inputs
from oracle import richardson
from conftest import read_golden


# ----------------------------------------------------------------- basis -----
def test_table1_basis_and_walk():
    """Table 1 (Sec. 3.1) and the successor walk 0011->0101->...->1100 of Sec. 3.1."""
    rows = read_golden("table1_basis_c4_2.txt")
    expect = [int(r[1]) for r in rows]
    assert list(oracle.basis(4, 2)) == expect
    walk = [3]
    while walk[-1] != 12:
        walk.append(oracle.next_state(walk[-1]))
    assert walk == expect


def test_hash_examples():
    """Sec. 3.2: f(0011)=1, f(1001)=4, f(1100)=6."""
    for bits, f in read_golden("hash_examples.txt"):
        assert oracle.hash_index(int(bits, 2)) == int(f)


@pytest.mark.parametrize("omega", range(1, 17))
def test_basis_brute_force(omega):
    """The successor enumerates exactly the popcount-N words, ascending."""
    words = np.arange(1 << omega, dtype=np.uint64)
    pc = np.array([bin(int(w)).count("1") for w in words])
    for n in range(0, omega + 1):
        b = oracle.basis(omega, n)
        assert np.array_equal(b, words[pc == n])


def test_binomial_extended():
    """Eq. (extcmn) against math.comb, including the n < m extension to 0."""
    for n in range(0, 64):
        for m in range(0, 64):
            assert oracle.binom(n, m) == (math.comb(n, m) if m <= n else 0)


@pytest.mark.parametrize("omega,n", [(10, 5), (13, 4), (16, 8), (20, 3), (18, 17)])
def test_hash_is_position(omega, n):
    """f(basis[r]) = r + 1 for every state, and binary search finds it."""
    b = oracle.basis(omega, n)
    assert len(b) == math.comb(omega, n)
    idx = np.random.default_rng(0).choice(len(b), size=min(len(b), 300), replace=False)
    for r in idx:
        assert oracle.hash_index(int(b[r])) == r + 1
        assert oracle.search(b, int(b[r])) == r
    # a word with the wrong popcount is absent
    assert oracle.search(b, (1 << (n + 1)) - 1 if n + 1 <= omega else 0) == -1


def test_large_omega_extremes():
    """Rank of the first and last states at Omega = 62 (the paper's limit)."""
    for n in (1, 5, 31):
        lo = (1 << n) - 1
        hi = lo << (62 - n)
        assert oracle.hash_index(lo) == 1
        assert oracle.hash_index(hi) == math.comb(62, n)
        assert oracle.next_state(lo) == (lo ^ (1 << (n - 1))) | (1 << n)


# ---------------------------------------------------------------- matrix -----
def test_worked_matrix():
    """Sec. 3.3 worked example: e = 1..4, V = -0.2, 2 pairs in 4 orbits."""
    M = np.array([[float(v) for v in r] for r in read_golden("matrix_4_2_g02.txt")])
    e, G = pd_inputs.picket_fence(4, -0.2)
    D = oracle.dense_matrix(4, 2, e, G)
    assert np.allclose(D, M, rtol=0, atol=1e-14)
    assert abs(np.linalg.eigvalsh(D)[0] - 5.54800127098854) < 1e-12


def _kron_hamiltonian(e, G):
    """Brute force from Eq. (2) on the full 2^Omega space: hard-core boson
    operators per orbit built with Kronecker products (orbit p = bit p)."""
    omega = len(e)
    lower = np.array([[0.0, 0.0], [1.0, 0.0]])     # |0> -> |1>: pair creation
    num = np.diag([0.0, 1.0])
    eye = np.eye(2)

    def op(single, p):
        out = np.array([[1.0]])
        for q in reversed(range(omega)):          # highest orbit is the leftmost factor
            out = np.kron(out, single if q == p else eye)
        return out

    Pd = [op(lower, p) for p in range(omega)]
    H = np.zeros((1 << omega, 1 << omega))
    for i in range(omega):
        H += (2 * e[i] + G[i, i]) * op(num, i)
        for j in range(omega):
            if i != j:
                H += G[i, j] * Pd[i] @ Pd[j].T
    return H


@pytest.mark.parametrize("omega", [3, 5, 7, 8])
def test_matrix_brute_force(omega):
    """The scattering + binary search matrix equals Eq. (2) built from operators."""
    rng = np.random.default_rng(omega)
    e = rng.uniform(-3, 3, omega)
    A = rng.normal(size=(omega, omega))
    G = (A + A.T) / 2
    Hfull = _kron_hamiltonian(e, G)
    pc = np.array([bin(w).count("1") for w in range(1 << omega)])
    for n in range(omega + 1):
        sel = np.nonzero(pc == n)[0]
        ref = Hfull[np.ix_(sel, sel)]
        got = oracle.dense_matrix(omega, n, e, G)
        assert np.allclose(got, ref, rtol=0, atol=1e-12), (omega, n)


def test_symmetry_and_nnz_count():
    """<x,Hy> = <Hx,y>; each row has N(Omega-N) off-diagonal entries; total
    Omega!/((N-1)!(Omega-N-1)!) (Sec. 5.3)."""
    omega, n = 11, 4
    rng = np.random.default_rng(3)
    e = rng.uniform(-1, 1, omega)
    A = rng.uniform(0.1, 1.0, size=(omega, omega))
    G = -(A + A.T)
    M = oracle.dense_matrix(omega, n, e, G)
    assert np.allclose(M, M.T, rtol=0, atol=0)
    off = (M != 0).sum(axis=1) - 1
    assert np.all(off == n * (omega - n))
    total = math.factorial(omega) // (math.factorial(n - 1) * math.factorial(omega - n - 1))
    assert int(off.sum()) == total
    x, y = rng.normal(size=(2, len(M)))
    hx = oracle.hx(omega, n, e, G, x)
    hy = oracle.hx(omega, n, e, G, y)
    assert abs(x @ hy - hx @ y) < 1e-10 * np.abs(x @ hy)


def test_hx_rows_matches_full():
    omega, n = 14, 6
    e, G = pd_inputs.separable_noise(omega, seed=4)
    x = pd_inputs.random_vector(math.comb(omega, n), 5)
    full = oracle.hx(omega, n, e, G, x)
    rows = np.array([0, 7, 100, 2000, len(x) - 1])
    assert np.array_equal(oracle.hx_rows(omega, n, e, G, x, rows), full[rows])


def test_monopole():
    """Monopole_Min/Max are the extreme diagonal elements (worked example: 5.6 and 13.6)."""
    e, G = pd_inputs.picket_fence(4, -0.2)
    lo, hi, pos = oracle.monopole(4, 2, e, G)
    assert abs(lo - 5.6) < 1e-14 and abs(hi - 13.6) < 1e-14 and pos == 0


# --------------------------------------------------------------- Jacobi ------
def test_jacobi_vs_library():
    rng = np.random.default_rng(9)
    for n in (1, 2, 5, 17, 40):
        A = rng.normal(size=(n, n)); A = A + A.T
        w, V = oracle.jacobi(A)
        assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-12)
        assert np.allclose(A @ V, V * w, atol=1e-11)
        assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)


# --------------------------------------------------------------- Lanczos -----
@pytest.mark.parametrize("row", read_golden("table2_lapack_c16_8.txt"))
def test_table2_energies(row):
    """Table 2 to all 12 printed decimals with G rounded to single precision."""
    g, e_pd, e_lapack = float(row[0]), float(row[1]), float(row[2])
    e, G = pd_inputs.picket_fence(16, g, g_float32=True)
    r = oracle.lanczos_ground(16, 8, e, G, window=50, tol=1e-12)
    assert r["converged"]
    assert abs(r["e0"] - e_pd) <= 1.5e-12
    assert abs(r["e0"] - e_lapack) <= 1.5e-12


def test_worked_example_lanczos_dim_below_window():
    """dim = 6 < window: one Krylov space spans everything (breakdown reading)."""
    e, G = pd_inputs.picket_fence(4, -0.2)
    r = oracle.lanczos_ground(4, 2, e, G, window=50)
    assert abs(r["e0"] - 5.54800127098854) < 1e-12


def test_config_omega12_against_richardson_and_dense():
    """Omega=12, N=6 picket fence from 0, G=-0.5: Lanczos = Richardson = dense eigh."""
    omega, n, e, G = pd_inputs.workload("omega12_n6_picket")
    r = oracle.lanczos_ground(omega, n, e, G, window=50, tol=1e-13)
    rich = richardson.ground_energy(e, -0.5, n)
    w, V = np.linalg.eigh(oracle.dense_matrix(omega, n, e, G))
    k = 0
    assert abs(r["e0"] - rich) <= 1e-10 * abs(rich)
    assert abs(r["e0"] - w[k]) <= 1e-12 * abs(w[k])
    # eigenvector: Delta_vector = sum |v_a^2 - v_b^2| (Table 2 caption)
    assert np.sum(np.abs(r["vec"] ** 2 - V[:, k] ** 2)) < 1e-10
    # attractive G: Perron-Frobenius, the ground state has one sign
    v = r["vec"] * np.sign(r["vec"][0])
    assert np.all(v > 0)


@pytest.mark.parametrize("omega,n,eps,g", [(10, 4, 0.3, -0.5), (9, 3, -1.0, -0.25), (12, 6, 0.0, -1.0)])
def test_degenerate_closed_form(omega, n, eps, g):
    """All e_i = eps, constant G: E0 = 2 eps N + G N (Omega - N + 1)."""
    e = np.full(omega, eps)
    G = np.full((omega, omega), g)
    r = oracle.lanczos_ground(omega, n, e, G, window=30, tol=1e-13)
    assert abs(r["e0"] - (2 * eps * n + g * n * (omega - n + 1))) < 1e-11


def test_random_start_and_permutation_invariance():
    omega, n = 12, 5
    e, G = pd_inputs.separable_noise(omega, seed=11)
    ref = oracle.lanczos_ground(omega, n, e, G, tol=1e-13)["e0"]
    start = pd_inputs.splitmix_uniform(7, math.comb(omega, n))
    r = oracle.lanczos_ground(omega, n, e, G, start=start, window=20, tol=1e-13)
    assert abs(r["e0"] - ref) < 1e-11 * abs(ref)
    perm = np.random.default_rng(1).permutation(omega)
    rp = oracle.lanczos_ground(omega, n, e[perm], G[np.ix_(perm, perm)], tol=1e-13)
    assert abs(rp["e0"] - ref) < 1e-11 * abs(ref)
    # variational: E0 <= Monopole_Min
    assert ref <= oracle.monopole(omega, n, e, G)[0]


def test_dense_jacobi_ground_state():
    """Cyclic Jacobi on a full (dim 252) matrix agrees with restarted Lanczos."""
    omega, n = 10, 5
    e, G = pd_inputs.separable_noise(omega, seed=6)
    w, _ = oracle.jacobi(oracle.dense_matrix(omega, n, e, G))
    r = oracle.lanczos_ground(omega, n, e, G, window=25, tol=1e-13)
    assert abs(r["e0"] - w.min()) < 1e-11 * abs(w.min())


def test_mode1_single_krylov_space():
    """Mode = 1 (no restart): with a window >= dim the Ritz value is exact."""
    omega, n = 8, 3
    e, G = pd_inputs.separable_noise(omega, seed=2)
    r = oracle.lanczos_ground(omega, n, e, G, window=56, mode=1)
    assert abs(r["e0"] - np.linalg.eigvalsh(oracle.dense_matrix(omega, n, e, G))[0]) < 1e-11


def test_trivial_sectors():
    """N = 0 and N = Omega: dim 1, E0 = H_00."""
    e, G = pd_inputs.separable_noise(7, seed=3)
    assert oracle.lanczos_ground(7, 0, e, G)["e0"] == 0.0
    full = oracle.lanczos_ground(7, 7, e, G)["e0"]
    assert abs(full - sum(2 * e[i] + G[i, i] for i in range(7))) < 1e-13


# ------------------------------------------------------------- Richardson ----
@pytest.mark.parametrize("row", read_golden("table3_richardson_g04.txt"))
def test_table3_richardson(row):
    """Table 3: the PairDiag column with G = float32(-0.4) (rounded to 7 decimals),
    the Richardson column with G = -0.4 (one unit of the last printed digit)."""
    omega, n = int(row[0]), int(row[1])
    assert math.comb(omega, n) == int(row[2])
    e, _ = pd_inputs.picket_fence(omega, -0.4)
    e_f32 = richardson.ground_energy(e, float(np.float32(-0.4)), n)
    e_ex = richardson.ground_energy(e, -0.4, n)
    assert abs(e_f32 - float(row[3])) <= 0.5e-7 + 1e-12
    assert abs(e_ex - float(row[4])) <= 1.0e-7


def test_richardson_one_pair_secular_equation():
    """N = 1: the energy is the lowest root of 1 + G sum_i 1/(x_i - E) = 0,
    i.e. the lowest eigenvalue of diag(x) + G 11^T (a library eigensolve)."""
    e = np.array([0.0, 0.7, 1.1, 2.5, 3.0])
    for g in (-0.3, -1.5):
        ref = np.linalg.eigvalsh(np.diag(2 * e) + g * np.ones((5, 5)))[0]
        assert abs(richardson.ground_energy(e, g, 1) - ref) < 1e-12


@pytest.mark.parametrize("seed,g", [(3, -0.4), (4, -0.4), (5, -1.5), (6, -0.05)])
def test_richardson_random_levels_vs_dense(seed, g):
    """Constant G with unsorted levels drawn uniform in [-10, 10] (the level
    distribution of the Omega=32, N=16 workload, whose constant-G twin is a
    large-size GPU pin): the Richardson energy equals the lowest eigenvalue of the
    dense matrix of Eq. 2 (a library eigensolve), for weak and strong pairing."""
    omega, n = 12, 6
    e = np.random.default_rng(seed).uniform(-10.0, 10.0, omega)
    G = np.full((omega, omega), g)
    ref = np.linalg.eigvalsh(oracle.dense_matrix(omega, n, e, G))[0]
    assert abs(richardson.ground_energy(e, g, n) - ref) <= 1e-11 * max(1.0, abs(ref))


@pytest.mark.parametrize("m", [4, 8, 12])
def test_ritz_residual_equals_beta_times_last_component(m):
    """The identity the solver's early end of a cycle relies on: after m Lanczos
    steps with full reorthogonalisation (Algorithm 2), the residual of the
    lowest Ritz pair (theta, Q s) of the m x m tridiagonal matrix is
    beta_m |s_m|.  Checked on the dense matrix of Eq. 2 (Omega=10, N=5) with
    numpy's eigensolver for the small matrix."""
    omega, n = 10, 5
    e, G = pd_inputs.separable_noise(omega, seed=21)
    A = oracle.dense_matrix(omega, n, e, G)
    dim = A.shape[0]
    q = np.random.default_rng(3).standard_normal(dim)
    Q = [q / np.linalg.norm(q)]
    alpha, beta = [], []
    for i in range(m):
        p = A @ Q[i]
        a = Q[i] @ p
        p = p - a * Q[i] - (beta[-1] * Q[i - 1] if i > 0 else 0.0)
        for _ in range(2):                        # full reorthogonalisation, twice
            p = p - np.stack(Q).T @ (np.stack(Q) @ p)
        alpha.append(a)
        beta.append(np.linalg.norm(p))
        Q.append(p / beta[-1])
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    w, S = np.linalg.eigh(T)
    y = np.stack(Q[:m]).T @ S[:, 0]
    resid = np.linalg.norm(A @ y - w[0] * y)
    assert abs(resid - beta[-1] * abs(S[-1, 0])) <= 1e-10 * max(1.0, resid)


def test_hellmann_feynman_occupations_and_couplings():
    """The derivative of the ground-state energy of Eq. 2 with respect to a
    parameter is the expectation value of the operator that multiplies it
    (Hellmann-Feynman).  Central differences of the oracle's lowest eigenvalue
    (numpy eigh of the oracle's matrix) must therefore equal, computed from
    the basis bits and the ground state alone:
      dE0/de_p  = 2 <n_p>  (the occupation number 2<S+_p S-_p> of Sec. 4.3),
      dE0/dG_pp = <n_p>,
      dE0/dG_pq = <P_p^+ P_q + P_q^+ P_p> for a symmetric change of G_pq and G_qp.
    A missing factor 2 on e_p, a dropped G_pp or a hop weighted by the wrong
    element of G fails one of these; the occupations also sum to 2N."""
    omega, n = 8, 3
    e, G = pd_inputs.separable_noise(omega, seed=4)
    b = oracle.basis(omega, n)
    index = {int(s): i for i, s in enumerate(b)}

    def lowest(e_, G_):
        return np.linalg.eigh(oracle.dense_matrix(omega, n, e_, G_))

    w, V = lowest(e, G)
    assert w[1] - w[0] > 1e-3                   # a non-degenerate ground state
    v = V[:, 0]
    bits = ((b[:, None] >> np.arange(omega, dtype=np.uint64)) & np.uint64(1)).astype(bool)
    n_exp = np.array([np.sum(v[bits[:, p]] ** 2) for p in range(omega)])
    assert abs(2 * n_exp.sum() - 2 * n) < 1e-12

    h = 1e-4

    def deriv(change):
        ep, Gp = change(+h)
        em, Gm = change(-h)
        return (lowest(ep, Gp)[0][0] - lowest(em, Gm)[0][0]) / (2 * h)

    def shift_e(p):
        def f(t):
            e2 = e.copy(); e2[p] += t
            return e2, G
        return f

    def shift_G(p, q):
        def f(t):
            G2 = G.copy(); G2[p, q] += t
            if p != q:
                G2[q, p] += t
            return e, G2
        return f

    for p in range(omega):
        assert abs(deriv(shift_e(p)) - 2 * n_exp[p]) < 1e-7, p
        assert abs(deriv(shift_G(p, p)) - n_exp[p]) < 1e-7, p
    for p, q in [(0, 1), (2, 5), (3, 7), (6, 4)]:
        hop = 0.0
        for i, s in enumerate(b):
            s = int(s)
            if (s >> q) & 1 and not (s >> p) & 1:      # P_p^+ P_q: pair moves q -> p
                hop += v[index[s ^ (1 << q) ^ (1 << p)]] * v[i]
        assert abs(deriv(shift_G(p, q)) - 2 * hop) < 1e-7, (p, q)

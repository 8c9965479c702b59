"""Odd-mass solves (blocking, Eq. 3) through the C ABI against the oracle, the
seniority formula and Richardson's equations."""
import math

import numpy as np
import pytest

import pd_inputs
from conftest import read_golden
from oracle import odd, richardson

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_2001_01978_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _opt(**kw):
    return pd.pairdiag_default_options(**kw)


def test_every_blocked_subspace_matches_the_oracle_fp64():
    omega, n = 12, 5
    e, G = pd_inputs.separable_noise(omega, seed=7)
    ref = odd.blocked_ground(omega, n, e, G, tol=1e-13)
    r = pd.pairdiag_odd_ground_state(omega, n, e, G, 1e-12, block=-1, opt=_opt(window=30))
    assert r["status"] == pd.PD_OK
    assert np.all(np.abs(r["energies"] - ref["energies"]) <= 1e-10 * np.abs(ref["energies"]))
    assert r["block"] == ref["block"]
    assert abs(r["e0"] - ref["e0"]) <= 1e-10 * abs(ref["e0"])
    assert r["occ"][r["block"]] == 1.0
    assert np.allclose(r["occ"], ref["occ"], atol=1e-8)
    assert abs(r["occ"].sum() - (2 * n + 1)) <= 1e-10
    assert r["vec"].shape == (math.comb(omega - 1, n),)
    assert np.sum(np.abs(r["vec"] ** 2 - ref["vec"] ** 2)) < 1e-8          # Delta_vector, Table 2 caption
    assert r["dim"] == math.comb(omega - 1, n)


def test_one_blocked_subspace_mixed():
    omega, n, b = 16, 7, 5
    e, G = pd_inputs.separable_noise(omega, seed=8)
    ref = odd.blocked_ground(omega, n, e, G, block=b, tol=1e-13)
    r = pd.pairdiag_odd_ground_state(omega, n, e, G, 1e-10, block=b, opt=_opt(precision=pd.PD_PREC_MIXED))
    assert r["status"] == pd.PD_OK and r["block"] == b
    assert abs(r["e0"] - ref["e0"]) <= 1e-8 * abs(ref["e0"])
    assert np.isnan(r["energies"]).sum() == omega - 1 and not np.isnan(r["energies"][b])
    assert np.allclose(r["occ"], ref["occ"], atol=1e-6)


@pytest.mark.parametrize("omega,n", [(20, 9), (13, 12), (11, 0)])
def test_degenerate_level_seniority_formula(omega, n):
    eps, g = 0.4, -0.25
    e = np.full(omega, eps)
    G = np.full((omega, omega), g)
    r = pd.pairdiag_odd_ground_state(omega, n, e, G, 1e-12)
    exact = eps * (2 * n + 1) + g * n * (omega - n)
    assert r["status"] == pd.PD_OK
    assert np.all(np.abs(r["energies"] - exact) <= 1e-10 * abs(exact))
    assert abs(r["occ"].sum() - (2 * n + 1)) <= 1e-9


def test_constant_g_blocked_orbits_match_richardson():
    """C(25,12) = 5.2e6 per subspace, all 26 subspaces, FP64."""
    omega, n, g = 26, 12, -0.4
    e = np.arange(1.0, omega + 1.0) + 0.013 * np.sin(np.arange(omega))
    G = np.full((omega, omega), g)
    r = pd.pairdiag_odd_ground_state(omega, n, e, G, 1e-11, want_vector=False)
    assert r["status"] == pd.PD_OK
    for b in range(omega):
        ref = e[b] + richardson.ground_energy(np.delete(e, b), g, n)
        assert abs(r["energies"][b] - ref) <= 1e-9 * abs(ref), b
    assert r["block"] == int(np.argmin(r["energies"]))


def test_filled_and_empty_pair_spaces():
    omega = 9
    e, G = pd_inputs.separable_noise(omega, seed=9)
    r = pd.pairdiag_odd_ground_state(omega, 0, e, G, 1e-12)
    assert r["block"] == int(np.argmin(e)) and r["e0"] == e.min()
    assert np.array_equal(r["occ"], (np.arange(omega) == r["block"]).astype(float))
    r = pd.pairdiag_odd_ground_state(omega, omega - 1, e, G, 1e-12)
    full = np.array([e[b] + sum(2 * e[i] + G[i, i] for i in range(omega) if i != b) for b in range(omega)])
    assert np.allclose(r["energies"], full, rtol=0, atol=1e-12 * np.abs(full).max())
    assert r["block"] == int(np.argmin(full))
    assert np.allclose(r["occ"], np.where(np.arange(omega) == r["block"], 1.0, 2.0))


def test_learned_start_gives_the_same_energies():
    omega, n = 12, 5
    e, G = pd_inputs.separable_noise(omega, seed=10)
    ref = odd.blocked_ground(omega, n, e, G, tol=1e-13)
    m = pd.pairdiag_mlp_create(3)
    try:
        r = pd.pairdiag_odd_ground_state(omega, n, e, G, 1e-12, opt=_opt(start=pd.PD_START_MLP), mlp=m)
    finally:
        pd.pairdiag_mlp_destroy(m)
    assert r["status"] == pd.PD_OK
    assert np.all(np.abs(r["energies"] - ref["energies"]) <= 1e-10 * np.abs(ref["energies"]))


def test_missed_tolerance_still_fills_the_outputs():
    omega, n = 12, 5
    e, G = pd_inputs.separable_noise(omega, seed=11)
    r = pd.pairdiag_odd_ground_state(omega, n, e, G, 1e-14, opt=_opt(window=4, max_restarts=2))
    assert r["status"] == pd.PD_ENOCONV
    assert np.all(np.isfinite(r["energies"])) and r["e0"] == r["energies"].min()
    assert 0 <= r["block"] < omega and r["occ"][r["block"]] == 1.0


def test_full_size_subspace_matches_the_oracle():
    """The odd-mass benchmark workload (25 orbits, 12 pairs + 1 particle, separable
    G, seed 1): the subspace of orbit 11, C(24,12) = 2.7e6 states, in both forms,
    against the oracle's E_b written by tests/golden/make_golden.py."""
    row = read_golden("omega25_n12_sepnoise_s1_odd_b11_e0.txt")[0]
    ref = float(row[0])
    assert int(row[1]) == 1
    e, G = pd_inputs.separable_noise(25, seed=1)
    r = pd.pairdiag_odd_ground_state(25, 12, e, G, 1e-10, block=11, want_vector=False)
    assert r["status"] == pd.PD_OK and r["block"] == 11
    assert abs(r["e0"] - ref) <= 1e-10 * abs(ref)
    r = pd.pairdiag_odd_ground_state(25, 12, e, G, 1e-9, block=11, want_vector=False,
                                     opt=_opt(precision=pd.PD_PREC_MIXED))
    assert r["status"] == pd.PD_OK
    assert abs(r["e0"] - ref) <= 1e-8 * abs(ref)

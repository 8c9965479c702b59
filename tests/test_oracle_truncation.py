"""Pins of the truncated-space oracle, Sec. 3.5 (CPU only)."""
import types
from pathlib import Path

import numpy as np
import pytest

import oracle
import pd_inputs
from oracle import truncation


def _problem(omega=12, seed=3):
    return pd_inputs.separable_noise(omega, seed=seed)


def test_no_truncation_when_the_limit_covers_the_space():
    omega, n = 10, 5
    e, G = _problem(10)
    t = truncation.truncate(omega, n, e, G, limit=252)
    assert not t["truncated"] and np.array_equal(t["kept"], oracle.basis(omega, n))
    ref = oracle.lanczos_ground(omega, n, e, G, tol=1e-13)["e0"]
    assert abs(truncation.ground_energy(omega, n, e, G, 252) - ref) <= 1e-11 * abs(ref)


def test_kept_states_are_those_with_the_lowest_diagonals():
    omega, n, limit = 12, 6, 300
    e, G = _problem()
    b = oracle.basis(omega, n)
    d = truncation.diagonals(omega, n, e, G, b)
    t = truncation.truncate(omega, n, e, G, limit)
    keep = np.isin(b, t["kept"])
    assert np.all(np.diff(t["kept"].astype(np.int64)) > 0)           # basis order
    assert d[keep].max() <= d[~keep].min()
    assert t["dim"] >= limit
    idx, cut = truncation.cutoff_bin(d, limit)
    assert np.count_nonzero(idx < cut) < limit <= np.count_nonzero(idx <= cut)
    # the same set as an exact sort of the diagonal (ties share a bin)
    order = np.argsort(d, kind="stable")
    assert set(b[order[:t["dim"]]].tolist()) == set(t["kept"].tolist())


def test_coarse_histogram_keeps_whole_bins():
    omega, n, limit = 12, 6, 100
    e, G = _problem()
    b = oracle.basis(omega, n)
    d = truncation.diagonals(omega, n, e, G, b)
    idx, cut = truncation.cutoff_bin(d, limit, bins=8)
    t = truncation.truncate(omega, n, e, G, limit, bins=8)
    assert t["dim"] == np.count_nonzero(idx <= cut) > limit
    assert set(t["kept"].tolist()) == set(b[idx <= cut].tolist())


def test_truncated_product_is_the_principal_submatrix():
    omega, n = 10, 5
    e, G = _problem(10, seed=4)
    t = truncation.truncate(omega, n, e, G, limit=120)
    b = oracle.basis(omega, n)
    pos = np.searchsorted(b, t["kept"])
    M = oracle.dense_matrix(omega, n, e, G)[np.ix_(pos, pos)]
    x = pd_inputs.random_vector(t["dim"], 5)
    assert np.allclose(truncation.hx_sub(omega, e, G, t["kept"], x), M @ x, rtol=0, atol=1e-12)
    # every kept state is found by the binary search at its position
    for j, s in enumerate(t["kept"][:50]):
        assert oracle.search(t["kept"], int(s)) == j


def test_interlacing_and_nesting():
    """Each truncated matrix is a principal submatrix of the next larger one, so
    the lowest eigenvalue can only fall as the limit grows, down to the exact E0."""
    omega, n = 12, 6
    e, G = _problem()
    full = oracle.lanczos_ground(omega, n, e, G, tol=1e-13)["e0"]
    prev_kept, prev_e = None, np.inf
    for limit in (40, 150, 400, 924):
        t = truncation.truncate(omega, n, e, G, limit)
        e0 = truncation.ground_energy(omega, n, e, G, limit)
        assert e0 >= full - 1e-10 * abs(full)
        assert e0 <= prev_e + 1e-10 * abs(full)
        if prev_kept is not None:
            assert set(prev_kept.tolist()) <= set(t["kept"].tolist())
        prev_kept, prev_e = t["kept"], e0
    assert abs(prev_e - full) <= 1e-10 * abs(full)


def test_limit_one_keeps_the_lowest_diagonal_state():
    omega, n = 10, 5
    e, G = _problem(10, seed=6)
    t = truncation.truncate(omega, n, e, G, limit=1)
    lo, _, pos = oracle.monopole(omega, n, e, G)
    assert t["dim"] == 1 and int(t["kept"][0]) == int(oracle.basis(omega, n)[pos])
    assert abs(truncation.ground_energy(omega, n, e, G, 1) - lo) <= 1e-12 * abs(lo)


def test_weak_pairing_tolerates_more_truncation():
    """Sec. 5.4: at the same truncation level the energy error grows with |G|
    (picket fence, constant G, C(12,6) kept to 30 %)."""
    omega, n, limit = 12, 6, 277
    errs = []
    for g in (-0.2, -0.4, -0.6):
        e, G = pd_inputs.picket_fence(omega, g)
        full = oracle.lanczos_ground(omega, n, e, G, tol=1e-13)["e0"]
        errs.append((truncation.ground_energy(omega, n, e, G, limit) - full) / abs(full))
    assert 0.0 < errs[0] < errs[1] < errs[2]


# ---- planted mistakes --------------------------------------------------------

TRUNC_MUTATIONS = {
    "drops_the_cutoff_bin": ("kept = b[idx <= cut]", "kept = b[idx < cut]"),
    "keeps_the_highest": ("idx = np.minimum(idx, bins - 1)", "idx = bins - 1 - np.minimum(idx, bins - 1)"),
}


def _mutant(old, new):
    src = Path(truncation.__file__).read_text()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle._trunc_mutant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), "trunc_mutant.py", "exec"), mod.__dict__)
    return mod


def _pins_hold(mod) -> bool:
    omega, n, limit = 12, 6, 300
    e, G = _problem()
    b = oracle.basis(omega, n)
    d = mod.diagonals(omega, n, e, G, b)
    t = mod.truncate(omega, n, e, G, limit)
    keep = np.isin(b, t["kept"])
    return bool(t["dim"] >= limit and d[keep].max() <= d[~keep].min())


def test_unmutated_truncation_passes():
    assert _pins_hold(truncation)


@pytest.mark.parametrize("name", sorted(TRUNC_MUTATIONS))
def test_planted_truncation_mistake_is_caught(name):
    assert not _pins_hold(_mutant(*TRUNC_MUTATIONS[name]))

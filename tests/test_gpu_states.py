"""The lowest few eigenpairs (locking, Sec. 3.4) through the C ABI against the
oracle's dense spectrum and the quasispin spectrum of a degenerate level."""
import math

import numpy as np
import pytest

import oracle
import pd_inputs
from oracle import excited

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_2001_01978_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def lowest(omega, n, e, G, k, tol, **opt):
    with pd.Solver(omega, n, e, G, **opt) as s:
        dim = pd.pairdiag_dim(s.h)
        vecs = torch.empty(k * dim, dtype=torch.float64, device="cuda")
        r = pd.pairdiag_lowest_states_dev(s.h, k, tol, vecs)
        g = s.ground_state(tol, want_vector=False)
        return r, vecs.view(k, dim).cpu().numpy(), g


def test_lowest_states_fp64_match_the_dense_spectrum():
    omega, n, k = 10, 5, 6
    e, G = pd_inputs.separable_noise(omega, seed=12)
    w, V = excited.lowest_k(omega, n, e, G, k)
    r, X, g = lowest(omega, n, e, G, k, 1e-12, window=30)
    assert r["status"] == pd.PD_OK
    scale = np.abs(w).max()
    assert np.allclose(r["energies"], w, rtol=0, atol=1e-10 * scale)
    assert np.allclose(X @ X.T, np.eye(k), atol=1e-9)
    gaps = np.diff(np.r_[-np.inf, w, np.inf])
    for j in range(k):
        if min(gaps[j], gaps[j + 1]) > 1e-4:
            assert abs(abs(X[j] @ V[:, j]) - 1.0) < 1e-8, j
    # the handle's ground state afterwards covers the whole space again
    assert abs(g["e0"] - w[0]) <= 1e-10 * scale


def test_degenerate_level_yields_each_copy():
    """Quasispin levels: one state at t = 0, then Omega - 1 = 9 copies at t = 1."""
    omega, n, eps, g, k = 10, 4, 0.5, -0.3, 6
    e = np.full(omega, eps)
    G = np.full((omega, omega), g)
    r, X, _ = lowest(omega, n, e, G, k, 1e-12)
    e0 = 2 * eps * n + g * n * (omega - n + 1)
    e1 = 2 * eps * n + g * (n * (omega - n + 1) - omega)
    ref = np.array([e0] + [e1] * (k - 1))
    assert np.allclose(r["energies"], ref, rtol=0, atol=1e-10 * abs(e0))
    assert np.allclose(X @ X.T, np.eye(k), atol=1e-9)
    for j in range(k):                                  # every vector an eigenvector of H
        y = oracle.hx(omega, n, e, G, X[j])
        assert np.linalg.norm(y - ref[j] * X[j]) <= 1e-8 * abs(ref[j])


def test_lowest_states_mixed_form():
    omega, n, k = 14, 7, 3
    e, G = pd_inputs.separable_noise(omega, seed=13)
    w, V = excited.lowest_k(omega, n, e, G, k)
    r, X, _ = lowest(omega, n, e, G, k, 1e-10, precision=pd.PD_PREC_MIXED)
    assert r["status"] == pd.PD_OK
    assert np.allclose(r["energies"], w, rtol=1e-8, atol=0)
    assert np.allclose(X @ X.T, np.eye(k), atol=1e-7)
    assert all(i["converged"] == 1 for i in r["info"])


def test_single_state_is_the_ground_state_and_bad_k_is_rejected():
    omega, n = 9, 4
    e, G = pd_inputs.separable_noise(omega, seed=14)
    with pd.Solver(omega, n, e, G) as s:
        r1 = pd.pairdiag_lowest_states_dev(s.h, 1, 1e-12)
        g = s.ground_state(1e-12, want_vector=False)
        assert abs(r1["energies"][0] - g["e0"]) <= 1e-10 * abs(g["e0"])
        for k in (0, math.comb(omega, n) + 1, 65):
            with pytest.raises(pd.PairDiagError) as err:
                pd.pairdiag_lowest_states_dev(s.h, k, 1e-12)
            assert err.value.code == pd.PD_EINVAL


def test_degenerate_level_full_size_omega24():
    """Omega=24, N=12 (dim 2.7e6) on one degenerate level, mixed form: the lowest
    three states are the quasispin level t = 0 and two copies of t = 1,
    E_t = 2 eps N + g [N (Omega - N + 1) - t (Omega + 1 - t)] (a closed form, so
    this pins the locking path at a size where the window leaves L2); the
    returned vectors are orthonormal."""
    omega, n, eps, g = 24, 12, 0.3, -0.25
    e = np.full(omega, eps)
    G = np.full((omega, omega), g)
    dim = math.comb(omega, n)
    with pd.Solver(omega, n, e, G, precision=pd.PD_PREC_MIXED, window=20) as s:
        vecs = torch.empty(3 * dim, dtype=torch.float64, device="cuda")
        r = pd.pairdiag_lowest_states_dev(s.h, 3, 1e-9, vecs)
        V = vecs.view(3, dim)
        gram = (V @ V.T).cpu().numpy()
    assert r["status"] == pd.PD_OK
    E = lambda t: 2 * eps * n + g * (n * (omega - n + 1) - t * (omega + 1 - t))
    expect = [E(0), E(1), E(1)]
    assert np.allclose(r["energies"], expect, rtol=1e-8, atol=0), (r["energies"], expect)
    assert np.allclose(gram, np.eye(3), atol=1e-7)

"""The truncated model space of Sec. 3.5 on the GPU (pairdiag_truncate) against
oracle/truncation.py: the kept states bit for bit, the truncated H*x row by
row, the truncated ground state, and the nonzero count of the truncated
matrix."""
import math

import numpy as np
import pytest

import oracle
import pd_inputs
from helpers import EPS32, EPS64, hx_bound
from oracle import truncation

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_2001_01978_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _kept_states(h):
    """Kept states of a truncated handle: the full basis where the map is >= 0,
    and the map itself (kept indices 0, 1, ... in basis order)."""
    full = pd.pairdiag_full_dim(h)
    m = torch.empty(full, dtype=torch.int32, device="cuda")
    pd.pairdiag_kept_map_dev(h, m)
    mp = m.cpu().numpy()
    keep = mp >= 0
    assert np.array_equal(mp[keep], np.arange(np.count_nonzero(keep)))
    return pd.pairdiag_basis(h)[keep]


# (omega, n, limit, bins): the paper's 10^8 bins, coarse bins (ties in the cut
# bin), a limit of one state, a block split with L = 12 over several blocks
KEPT_CASES = [(12, 6, 300, 0), (14, 7, 1000, 0), (16, 8, 5000, 100), (16, 5, 1, 0), (13, 4, 200, 7),
              (18, 9, 20000, 0), (20, 6, 4000, 1000), (17, 16, 5, 0)]


@pytest.mark.parametrize("omega,n,limit,bins", KEPT_CASES)
def test_kept_states_bit_exact(omega, n, limit, bins):
    e, G = pd_inputs.separable_noise(omega, seed=omega * 7 + n)
    ref = truncation.truncate(omega, n, e, G, limit, bins or truncation.DEFAULT_BINS)
    with pd.Solver(omega, n, e, G) as s:
        kept = pd.pairdiag_truncate(s.h, limit, bins)
        assert kept == ref["dim"] == s.dim
        assert np.array_equal(_kept_states(s.h), ref["kept"])
        assert pd.pairdiag_full_dim(s.h) == math.comb(omega, n)


def test_no_truncation_cases():
    """limit >= C(Omega,N), an equal diagonal everywhere, and limit 0 (restore)
    leave the full space: no map, the full dimension."""
    omega, n = 12, 6
    e, G = pd_inputs.separable_noise(omega, seed=3)
    with pd.Solver(omega, n, e, G) as s:
        assert pd.pairdiag_truncate(s.h, 924) == 924
        with pytest.raises(pd.PairDiagError):
            pd.pairdiag_kept_map_dev(s.h, torch.empty(924, dtype=torch.int32, device="cuda"))
        assert pd.pairdiag_truncate(s.h, 100) < 924
        assert pd.pairdiag_truncate(s.h, 0) == 924 == s.dim
    e, G = pd_inputs.picket_fence(omega, -0.3)
    e[:] = 1.5                                     # degenerate level: every diagonal element equal
    with pd.Solver(omega, n, e, G) as s:
        assert pd.pairdiag_truncate(s.h, 10) == 924
        assert truncation.truncate(omega, n, e, G, 10)["dim"] == 924


@pytest.mark.parametrize("omega,n,limit,low", [(12, 6, 300, 0), (16, 8, 4000, 0), (18, 7, 10000, 9),
                                                (20, 10, 60000, 0), (17, 3, 100, 0)])
def test_truncated_hx_vs_oracle(omega, n, limit, low):
    """Both precisions, element by element against the oracle's H x on the kept
    states (binary search per hop) under the rounding bound of each row."""
    e, G = pd_inputs.separable_noise(omega, seed=omega + 50 * n)
    ref_t = truncation.truncate(omega, n, e, G, limit)
    kept = ref_t["kept"]
    x = pd_inputs.random_vector(len(kept), 11)
    y_ref = truncation.hx_sub(omega, e, G, kept, x)
    Gabs = np.abs(G)
    d = 2.0 * np.asarray(e) + np.diag(G)
    e_abs = (np.abs(d) - np.diag(Gabs)) / 2.0
    scale = truncation.hx_sub(omega, e_abs, Gabs, kept, np.abs(x))
    with pd.Solver(omega, n, e, G, low_bits=low) as s:
        assert pd.pairdiag_truncate(s.h, limit) == len(kept)
        y = pd.pairdiag_hx(s.h, x)
        assert np.all(np.abs(y - y_ref) <= hx_bound(omega, n, scale, EPS64))
        x32 = torch.from_numpy(x.astype(np.float32)).cuda()
        y32 = torch.empty_like(x32)
        pd.pairdiag_hx_dev(s.h, pd.PD_PREC_MIXED, x32, y32)
        torch.cuda.synchronize()
        y_ref32 = truncation.hx_sub(omega, e, G, kept, x.astype(np.float32).astype(np.float64))
        # FP32 G and d, FP32 row sums
        assert np.all(np.abs(y32.cpu().numpy() - y_ref32) <= hx_bound(omega, n, scale, EPS32))


def test_truncated_nnz():
    """pairdiag_nnz of a truncated handle = the off-diagonal nonzeros of the
    principal submatrix (the oracle's matrix with every G_ij = 1)."""
    omega, n, limit = 12, 6, 250
    e, G = pd_inputs.separable_noise(omega, seed=5)
    kept = truncation.truncate(omega, n, e, G, limit)["kept"]
    M = truncation.sub_matrix(omega, e, np.ones((omega, omega)), kept)
    nnz_ref = int(np.count_nonzero(M - np.diag(np.diag(M))))
    with pd.Solver(omega, n, e, G) as s:
        pd.pairdiag_truncate(s.h, limit)
        assert pd.pairdiag_nnz(s.h) == nnz_ref
        pd.pairdiag_truncate(s.h, 0)
        assert pd.pairdiag_nnz(s.h) == 924 * 36


@pytest.mark.parametrize("precision,rel,start", [(0, 1e-10, pd.PD_START_RANDOM), (0, 1e-10, pd.PD_START_HF),
                                                 (1, 1e-8, pd.PD_START_FIRST)])
def test_truncated_ground_state_nested(precision, rel, start):
    """Truncated E0 against the lowest eigenvalue of the oracle's principal
    submatrix (dense) for nested limits; E0 falls as the limit grows (Cauchy
    interlacing) and reaches the full E0 (Sec. 5.4 studies this convergence)."""
    omega, n = 12, 6
    e, G = pd_inputs.separable_noise(omega, seed=8)
    full = oracle.lanczos_ground(omega, n, e, G, tol=1e-13)["e0"]
    last = np.inf
    with pd.Solver(omega, n, e, G, precision=precision, start=start, window=30) as s:
        for limit in (20, 100, 400, 924):
            pd.pairdiag_truncate(s.h, limit)
            r = s.ground_state(1e-12 if precision == 0 else 1e-9)
            assert r["status"] == pd.PD_OK
            ref = truncation.ground_energy(omega, n, e, G, limit) if limit < 924 else full
            assert abs(r["e0"] - ref) <= rel * abs(ref), (limit, r["e0"], ref)
            assert r["e0"] <= last + 1e-9 * abs(ref)
            last = r["e0"]
            assert len(r["vec"]) == s.dim
        assert abs(last - full) <= rel * abs(full)


def test_truncated_omega20_eigenpair_and_occupations():
    """Omega=20, N=10 (dim 184,756) truncated to about 30,000 states: the kept
    set bit for bit; the returned vector is an eigenvector of the oracle's
    truncated operator (Rayleigh quotient = E0, residual <= 1e-9 |E0|); the
    occupation numbers of that vector against the oracle's basis bits."""
    omega, n, limit = 20, 10, 30000
    e, G = pd_inputs.separable_noise(omega, seed=20)
    ref = truncation.truncate(omega, n, e, G, limit)
    kept = ref["kept"]
    with pd.Solver(omega, n, e, G, precision=pd.PD_PREC_FP64, window=30) as s:
        assert pd.pairdiag_truncate(s.h, limit) == len(kept)
        assert np.array_equal(_kept_states(s.h), kept)
        v = torch.empty(s.dim, dtype=torch.float64, device="cuda")
        r = pd.pairdiag_ground_state_dev(s.h, 1e-11, v)
        assert r["status"] == pd.PD_OK
        occ = pd.pairdiag_occupations_dev(s.h, v, omega)
        vh = v.cpu().numpy()
    w = truncation.hx_sub(omega, e, G, kept, vh)
    lam = float(vh @ w) / float(vh @ vh)
    assert abs(lam - r["e0"]) <= 1e-11 * abs(lam)
    assert np.linalg.norm(w - lam * vh) / np.linalg.norm(vh) <= 1e-9 * abs(lam)
    bits = ((kept[:, None] >> np.arange(omega, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)
    occ_ref = 2.0 * (vh * vh) @ bits
    assert np.allclose(occ, occ_ref, rtol=0, atol=1e-12)
    assert abs(occ.sum() - 2 * n) <= 1e-10

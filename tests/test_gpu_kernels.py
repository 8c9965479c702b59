"""GPU parity of the basis, ranking, H*x and reduction kernels against the CPU
oracle, through the C ABI."""
import math

import numpy as np
import pytest

import oracle
import pd_inputs
from conftest import read_golden
from helpers import EPS32, EPS64, abs_row_scale, hx_bound

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_2001_01978_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    pd.lib()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _solver(omega, n, e=None, G=None, **opt):
    if e is None:
        e, G = pd_inputs.separable_noise(omega, seed=omega * 100 + n)
    return pd.Solver(omega, n, e, G, **opt), e, G


# ------------------------------------------------------------------ basis ---
@pytest.mark.parametrize("omega", range(1, 25))
def test_basis_bit_exact_small(omega):
    """Every (Omega <= 24, N): the whole GPU basis equals the oracle's, word for word."""
    for n in range(omega + 1):
        s, _, _ = _solver(omega, n)
        with s:
            got = pd.pairdiag_basis(s.h)
        assert np.array_equal(got, oracle.basis(omega, n)), (omega, n)


def test_basis_table1():
    rows = read_golden("table1_basis_c4_2.txt")
    s, _, _ = _solver(4, 2)
    with s:
        assert list(pd.pairdiag_basis(s.h)) == [int(r[1]) for r in rows]


@pytest.mark.parametrize("omega,n", [(24, 12), (30, 15), (32, 16), (40, 6), (62, 3)])
def test_basis_sampled_large(omega, n):
    """Chunks of the basis at random offsets: ascending, right popcount, and the
    paper's hash of each word (oracle) equals its position + 1."""
    e, G = pd_inputs.separable_noise(omega, seed=1)
    dim = math.comb(omega, n)
    rng = np.random.default_rng(omega)
    with pd.Solver(omega, n, e, G) as s:
        for first in [0, dim - 3000] + [int(v) for v in rng.integers(0, dim - 3000, size=3)]:
            first = max(0, first)
            cnt = min(3000, dim - first)
            out = torch.empty(cnt, dtype=torch.int64, device="cuda")
            pd.pairdiag_basis_dev(s.h, first, cnt, out)
            w = out.cpu().numpy().view(np.uint64)
            assert np.all(w[1:] > w[:-1])
            for j in range(0, cnt, 97):
                assert bin(int(w[j])).count("1") == n
                assert oracle.hash_index(int(w[j])) == first + j + 1


def _random_states(omega, n, count, seed):
    """Uniformly random Omega-bit words with n set bits (numpy, no ranking)."""
    rng = np.random.default_rng(seed)
    words = np.zeros(count, dtype=np.uint64)
    for i in range(count):
        for p in rng.choice(omega, size=n, replace=False):
            words[i] |= np.uint64(1) << np.uint64(int(p))
    return words


@pytest.mark.parametrize("omega,n", [(12, 6), (20, 9), (24, 12), (32, 16), (38, 10), (44, 7), (50, 5), (62, 3), (62, 1)])
def test_rank_vs_oracle_hash(omega, n):
    """pairdiag_rank_dev on random states equals the oracle's hash f - 1 (Sec. 3.2),
    bit for bit, including the first and last states of the basis."""
    words = _random_states(omega, n, 4000, seed=omega * 64 + n)
    lo = (1 << n) - 1
    words[:2] = [lo, lo << (omega - n)]
    expect = np.array([oracle.hash_index(int(w)) - 1 for w in words], dtype=np.uint64)
    e, G = pd_inputs.separable_noise(omega, seed=2)
    h = pd.pairdiag_create(omega, n, e, G)
    try:
        states = torch.from_numpy(words.view(np.int64)).cuda()
        ranks = torch.empty_like(states)
        pd.pairdiag_rank_dev(h, states, ranks)
        got = ranks.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, expect), np.flatnonzero(got != expect)[:5]
    finally:
        pd.pairdiag_destroy(h)


@pytest.mark.parametrize("omega,n", [(20, 9), (32, 16), (50, 5)])
def test_rank_roundtrip(omega, n):
    e, G = pd_inputs.separable_noise(omega, seed=2)
    h = pd.pairdiag_create(omega, n, e, G)
    try:
        dim = math.comb(omega, n)
        r = np.random.default_rng(1).integers(0, dim, size=5000).astype(np.int64)
        r[:2] = [0, dim - 1]
        states = torch.empty(len(r), dtype=torch.int64, device="cuda")
        for i, ri in enumerate(r[:64]):
            pd.pairdiag_basis_dev(h, int(ri), 1, states[i:i + 1])
        ranks = torch.empty_like(states)
        pd.pairdiag_rank_dev(h, states[:64], ranks[:64])
        assert np.array_equal(ranks[:64].cpu().numpy(), r[:64])
        # words with the wrong popcount or beyond Omega bits are rejected
        bad = torch.tensor([0b111, (1 << omega) | 1], dtype=torch.int64, device="cuda")
        rb = torch.empty_like(bad)
        pd.pairdiag_rank_dev(h, bad, rb)
        assert np.all(rb.cpu().numpy().view(np.uint64) == np.uint64(2**64 - 1))
    finally:
        pd.pairdiag_destroy(h)


# -------------------------------------------------------------------- H x ---
def test_hx_worked_matrix_exact():
    M = np.array([[float(v) for v in r] for r in read_golden("matrix_4_2_g02.txt")])
    e, G = pd_inputs.picket_fence(4, -0.2)
    with pd.Solver(4, 2, e, G) as s:
        for j in range(6):
            x = np.zeros(6); x[j] = 1.0
            assert np.allclose(pd.pairdiag_hx(s.h, x), M[:, j], rtol=0, atol=2e-15)


HX_CASES = [
    (12, 6, 0), (14, 7, 0), (16, 5, 0), (18, 9, 0), (20, 10, 0), (22, 4, 0), (17, 1, 0), (17, 16, 0),
    (13, 6, 5), (15, 7, 8), (16, 8, 13), (19, 9, 3), (10, 0, 0), (10, 10, 0), (24, 12, 0), (26, 3, 0),
]


@pytest.mark.parametrize("omega,n,low", HX_CASES)
def test_hx_fp64_vs_oracle(omega, n, low):
    e, G = pd_inputs.separable_noise(omega, seed=omega + 31 * n)
    with pd.Solver(omega, n, e, G, low_bits=low) as s:
        x = pd_inputs.random_vector(s.dim, omega * 7 + n)
        b = oracle.basis(omega, n)
        ref = oracle.hx(omega, n, e, G, x, b)
        got = pd.pairdiag_hx(s.h, x)
        bound = hx_bound(omega, n, abs_row_scale(omega, n, e, G, x, basis=b), EPS64)
        assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / np.maximum(bound, 1e-300))


@pytest.mark.parametrize("omega,n,low", [c for c in HX_CASES if c[0] <= 22])
def test_hx_fp32_vs_oracle(omega, n, low):
    e, G = pd_inputs.separable_noise(omega, seed=omega + 31 * n)
    with pd.Solver(omega, n, e, G, low_bits=low) as s:
        x32 = pd_inputs.random_vector(s.dim, omega * 7 + n).astype(np.float32)
        xt = torch.from_numpy(x32).cuda()
        yt = torch.empty_like(xt)
        pd.pairdiag_hx_dev(s.h, pd.PD_PREC_MIXED, xt, yt)
        got = yt.cpu().numpy().astype(np.float64)
        x = x32.astype(np.float64)
        b = oracle.basis(omega, n)
        ref = oracle.hx(omega, n, e, G, x, b)
        bound = hx_bound(omega, n, abs_row_scale(omega, n, e, G, x, basis=b), EPS32)
        assert np.all(np.abs(got - ref) <= bound)


EPS_FF = 2.0 ** -44     # per term: float-float products and sums (about 2^-48), with margin


@pytest.mark.parametrize("omega,n,low", [(12, 6, 0), (16, 5, 0), (20, 10, 0), (22, 4, 0), (24, 12, 0),
                                         (17, 16, 0), (19, 9, 3), (10, 0, 0), (10, 10, 0), (18, 9, 13)])
def test_hx_floatfloat_vs_oracle(omega, n, low):
    """Float-float rows of an FP32 vector (the product the mixed form's FP64
    Rayleigh refinement takes) against the oracle's FP64 H*x of the same values,
    element by element, under a bound of 2^-44 per term of a row; FP32 row sums
    of the same vector miss that bound by orders of magnitude, so the test
    tells the two apart."""
    e, G = pd_inputs.separable_noise(omega, seed=omega + 31 * n + 5)
    with pd.Solver(omega, n, e, G, low_bits=low) as s:
        x32 = pd_inputs.random_vector(s.dim, omega * 11 + n).astype(np.float32)
        xt = torch.from_numpy(x32).cuda()
        yt = torch.empty(s.dim, dtype=torch.float64, device="cuda")
        pd.pairdiag_hx_dev(s.h, pd.PD_HX_FLOATFLOAT, xt, yt)
        got = yt.cpu().numpy()
        y32 = torch.empty_like(xt)
        pd.pairdiag_hx_dev(s.h, pd.PD_PREC_MIXED, xt, y32)
        got32 = y32.cpu().numpy().astype(np.float64)
    x = x32.astype(np.float64)
    b = oracle.basis(omega, n)
    ref = oracle.hx(omega, n, e, G, x, b)
    bound = hx_bound(omega, n, abs_row_scale(omega, n, e, G, x, basis=b), EPS_FF)
    assert np.all(np.abs(got - ref) <= bound), np.max(np.abs(got - ref) / np.maximum(bound, 1e-300))
    if s.dim > 100:
        assert np.any(np.abs(got32 - ref) > bound)


def test_hx_floatfloat_not_on_truncated_space():
    """The float-float product covers the full space only: a truncated handle
    answers PD_ENOTSUP (and its mixed solves refine with the FP64 product)."""
    e, G = pd_inputs.separable_noise(14, seed=3)
    with pd.Solver(14, 7, e, G) as s:
        pd.pairdiag_truncate(s.h, 1000)
        xt = torch.ones(s.dim, dtype=torch.float32, device="cuda")
        yt = torch.empty(s.dim, dtype=torch.float64, device="cuda")
        with pytest.raises(pd.PairDiagError) as ex:
            pd.pairdiag_hx_dev(s.h, pd.PD_HX_FLOATFLOAT, xt, yt)
        assert ex.value.code == pd.PD_ENOTSUP


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("omega,n,low", [(16, 5, 0), (20, 10, 0), (19, 9, 3), (15, 7, 8), (22, 4, 0), (24, 12, 13),
                                         (26, 3, 12), (21, 2, 9), (18, 16, 10), (12, 6, 12), (23, 1, 8), (20, 19, 11)])
def test_hx_variants_vs_oracle(omega, n, low, variant):
    """The five H*x kernel variants (neighbour blocks staged one at a time / all
    at once / gathered from global memory with O(1) hop tables, in lean loops or
    in deep gather groups, and the lean loops built for five CTAs per SM),
    including low and high filling, a single block
    (L = Omega) and N = 1, Omega - 1."""
    e, G = pd_inputs.separable_noise(omega, seed=omega + 7 * n)
    b = oracle.basis(omega, n)
    x = pd_inputs.random_vector(len(b), omega + n)
    ref = oracle.hx(omega, n, e, G, x, b)
    scale = abs_row_scale(omega, n, e, G, x, basis=b)
    with pd.Solver(omega, n, e, G, low_bits=low, hx_variant=variant) as s:
        got = pd.pairdiag_hx(s.h, x)
        assert np.all(np.abs(got - ref) <= hx_bound(omega, n, scale, EPS64))
        xt = torch.from_numpy(x.astype(np.float32)).cuda()
        yt = torch.empty_like(xt)
        pd.pairdiag_hx_dev(s.h, pd.PD_PREC_MIXED, xt, yt)
        x32 = x.astype(np.float32).astype(np.float64)
        ref32 = oracle.hx(omega, n, e, G, x32, b)
        scale32 = abs_row_scale(omega, n, e, G, x32, basis=b)
        assert np.all(np.abs(yt.cpu().numpy() - ref32) <= hx_bound(omega, n, scale32, EPS32))


def test_hx_dev_fp64_and_stream():
    omega, n = 20, 9
    e, G = pd_inputs.constant_noise(omega, seed=5)
    with pd.Solver(omega, n, e, G) as s:
        st = torch.cuda.Stream()
        pd.pairdiag_set_stream(s.h, st)
        x = torch.from_numpy(pd_inputs.random_vector(s.dim, 2)).cuda()
        y = torch.empty_like(x)
        with torch.cuda.stream(st):
            pd.pairdiag_hx_dev(s.h, pd.PD_PREC_FP64, x, y)
        st.synchronize()
        ref = oracle.hx(omega, n, e, G, x.cpu().numpy())
        assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
        # input validation is host-side
        with pytest.raises(pd.PairDiagError):
            pd.pairdiag_hx_dev(s.h, pd.PD_PREC_FP64, x, x)


@pytest.mark.parametrize("name", ["omega30_n15_sepnoise_s2", "omega32_n16_constnoise_s3"])
def test_hx_full_size_sampled(name):
    """Full-size workloads: sampled rows of the GPU product against the oracle
    row by row (binary search over the oracle's own basis)."""
    omega, n, e, G = pd_inputs.workload(name)
    b = oracle.basis(omega, n)
    with pd.Solver(omega, n, e, G) as s:
        dim = s.dim
        rows = np.sort(np.random.default_rng(7).choice(dim, size=400, replace=False))
        rows[:2] = [0, dim - 1]
        for prec, tdt, eps in ((pd.PD_PREC_MIXED, torch.float32, EPS32), (pd.PD_PREC_FP64, torch.float64, EPS64)):
            gen = torch.Generator(device="cuda").manual_seed(11)
            x = torch.randn(dim, dtype=tdt, device="cuda", generator=gen)
            y = torch.empty_like(x)
            pd.pairdiag_hx_dev(s.h, prec, x, y)
            torch.cuda.synchronize()
            xh = x.cpu().numpy().astype(np.float64)
            ref = oracle.hx_rows(omega, n, e, G, xh, rows, b)
            got = y.cpu().numpy()[rows].astype(np.float64)
            bound = hx_bound(omega, n, abs_row_scale(omega, n, e, G, xh, rows, b), eps)
            assert np.all(np.abs(got - ref) <= bound), (prec, np.max(np.abs(got - ref) / bound))
            del x, y


# ------------------------------------------------------- per-row reductions ---
@pytest.mark.parametrize("omega,n", [(4, 2), (12, 6), (18, 7), (24, 12)])
def test_monopole_vs_oracle(omega, n):
    e, G = pd_inputs.separable_noise(omega, seed=3)
    with pd.Solver(omega, n, e, G) as s:
        lo, hi, pos = pd.pairdiag_monopole(s.h)
    rlo, rhi, rpos = oracle.monopole(omega, n, e, G)
    assert lo == rlo and hi == rhi and pos == rpos


def test_occupations_sum_rule():
    omega, n = 16, 6
    e, G = pd_inputs.separable_noise(omega, seed=8)
    with pd.Solver(omega, n, e, G) as s:
        r = s.ground_state(1e-11)
        v = torch.from_numpy(r["vec"]).cuda()
        occ = pd.pairdiag_occupations_dev(s.h, v, omega)
    b = oracle.basis(omega, n)
    w = r["vec"] ** 2
    ref = np.array([2.0 * w[(b >> np.uint64(p)) & np.uint64(1) == 1].sum() for p in range(omega)])
    assert np.allclose(occ, ref, atol=1e-12)
    assert abs(occ.sum() - 2 * n) < 1e-10


# --------------------------------------------------------- vector algebra ---
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_multidot(dtype):
    tdt = getattr(torch, dtype)
    n, m = 1_000_003, 13
    g = torch.Generator(device="cuda").manual_seed(3)
    Q = torch.randn(m, n, dtype=tdt, device="cuda", generator=g)
    p = torch.randn(n, dtype=tdt, device="cuda", generator=g)
    e, G = pd_inputs.picket_fence(4, -0.2)
    with pd.Solver(4, 2, e, G) as s:
        got = pd.pairdiag_multidot(s.h, Q, n, m, p, n)
    ref = Q.double().cpu().numpy() @ p.double().cpu().numpy()
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("m", [1, 2, 3, 7, 20, 50, 64])
def test_tridiag_vs_jacobi(m):
    rng = np.random.default_rng(m)
    alpha = rng.normal(size=m) * 3
    beta = np.abs(rng.normal(size=m - 1)) + 0.01
    e, G = pd_inputs.picket_fence(4, -0.2)
    with pd.Solver(4, 2, e, G) as s:
        theta, svec = pd.pairdiag_tridiag_lowest(s.h, alpha, beta)
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    w, V = oracle.jacobi(T)
    order = np.argsort(w)
    assert abs(theta[0] - w[order[0]]) <= 1e-13 * max(1.0, np.abs(w).max())
    if m > 1:   # the second Ritz value is a gap estimate, bracketed in FP32
        assert abs(theta[1] - w[order[1]]) <= 1e-6 * max(1.0, np.abs(w).max())
    v = V[:, order[0]]
    assert abs(abs(v @ svec) - 1.0) < 1e-11
    assert np.linalg.norm(T @ svec - theta[0] * svec) < 1e-11 * max(1.0, np.abs(w).max())


def test_tridiag_clustered():
    """Nearly-degenerate lowest pair and tiny off-diagonals."""
    alpha = np.array([1.0, 1.0 + 1e-9, 5.0, 7.0])
    beta = np.array([1e-12, 0.5, 1e-30])
    e, G = pd_inputs.picket_fence(4, -0.2)
    with pd.Solver(4, 2, e, G) as s:
        theta, svec = pd.pairdiag_tridiag_lowest(s.h, alpha, beta)
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    w = np.linalg.eigvalsh(T)
    assert abs(theta[0] - w[0]) < 1e-14 and abs(theta[1] - w[1]) < 1e-5
    assert np.linalg.norm(T @ svec - theta[0] * svec) < 1e-12


# ---------------------------------------------------------------- autotuner ---
def test_autotune_records_fastest_schedule():
    omega, n = 18, 8
    e, G = pd_inputs.separable_noise(omega, seed=17)
    best, allc = pd.pairdiag_autotune(omega, n, e, G, pd.PD_PREC_MIXED, reps=3)
    assert allc and best["ms"] == min(c["ms"] for c in allc)
    assert {c["low_bits"] for c in allc} == set(range(8, 14))
    assert pd.pairdiag_tune_get(omega, n, pd.PD_PREC_MIXED) == (best["low_bits"], best["hx_variant"])
    # a handle created afterwards uses the recorded schedule and stays exact
    with pd.Solver(omega, n, e, G, precision=pd.PD_PREC_MIXED) as s:
        x = pd_inputs.random_vector(s.dim, 5)
        y = pd.pairdiag_hx(s.h, x)
    assert np.max(np.abs(y - oracle.hx(omega, n, e, G, x))) <= 1e-11 * np.max(np.abs(y))
    pd.pairdiag_tune_set(omega, n, pd.PD_PREC_MIXED, 0, 0)
    assert pd.pairdiag_tune_get(omega, n, pd.PD_PREC_MIXED) == (0, 0)

"""The learned warm start on the GPU: network kernels against the FP64 twin in
oracle/, the per-orbit target fit, the product start vector, and the gain of
the trained network over a random start."""
import math

import numpy as np
import pytest

import oracle
import pd_inputs
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_2001_01978_gb300")
from paper_2001_01978_gb300 import warmstart  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def _params(seed, scale=1.0):
    m = pd.pairdiag_mlp_create(seed)
    th = pd.pairdiag_mlp_get_params(m).astype(np.float64)
    rng = np.random.default_rng(seed)
    th[-129:] += rng.normal(0, 0.1, size=129)          # nonzero head and biases
    th *= scale
    pd.pairdiag_mlp_set_params(m, th.astype(np.float32))
    return m, pd.pairdiag_mlp_get_params(m).astype(np.float64)


@pytest.mark.parametrize("rows", [5, 64, 300, 1000])
def test_forward_and_gradient_vs_oracle(rows):
    """BF16 tensor-core forward/backward vs the FP64 twin evaluated on the same
    bfloat16-rounded inputs and weights (the remaining difference is FP32
    accumulation and the bfloat16 storage of backward intermediates)."""
    m, theta = _params(rows)
    rng = np.random.default_rng(rows + 1)
    X = rng.normal(size=(rows, 16)).astype(np.float32)
    t = rng.normal(size=rows).astype(np.float32)
    out = pd.pairdiag_mlp_forward(m, X)
    ref_out, _ = omlp.forward(theta, X.astype(np.float64), bf16_mode=True)
    assert np.max(np.abs(out - ref_out)) <= 1e-2 * max(1.0, np.max(np.abs(ref_out)))
    loss, grad = pd.pairdiag_mlp_loss_grad(m, X, t)
    ref_loss, ref_grad = omlp.loss_and_grad(theta, X.astype(np.float64), t.astype(np.float64), bf16_mode=True)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    for (name, lo, hi) in [("W1", 0, 2048), ("b1", 2048, 2176), ("W2", 2176, 18560), ("b2", 18560, 18688),
                           ("W3", 18688, 35072), ("b3", 35072, 35200), ("w4", 35200, 35328), ("b4", 35328, 35329)]:
        g, r = grad[lo:hi].astype(np.float64), ref_grad[lo:hi]
        assert np.linalg.norm(g - r) <= 3e-2 * np.linalg.norm(r) + 1e-7, name
    pd.pairdiag_mlp_destroy(m)


def test_training_reduces_loss():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(512, 16)).astype(np.float32)
    t = (np.tanh(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]).astype(np.float32)
    m = pd.pairdiag_mlp_create(1)
    hist = pd.pairdiag_mlp_train(m, X, t, 400, 2e-3)
    assert hist[-1] < 0.1 * hist[0]
    pd.pairdiag_mlp_destroy(m)


def test_product_fit_and_start_vs_numpy():
    """Target fit: weighted least squares of log|v| on the occupation bits (numpy
    lstsq on the oracle's basis and eigenvector); the product start vector."""
    omega, n = 12, 5
    e, G = pd_inputs.separable_noise(omega, seed=21)
    ref = oracle.lanczos_ground(omega, n, e, G, tol=1e-13)
    b = oracle.basis(omega, n)
    occ = ((b[:, None] >> np.arange(omega, dtype=np.uint64)) & np.uint64(1)).astype(np.float64)
    v = ref["vec"] * np.sign(ref["vec"][0])
    wgt = v * v
    # normal equations of the weighted fit, with the library's ridge of
    # 1e-9 * trace/omega (orbits that are almost always full or empty)
    M = occ.T @ (occ * wgt[:, None])
    rhs = occ.T @ (wgt * np.log(np.abs(v)))
    M += 1e-9 * np.trace(M) / omega * np.eye(omega)
    w_np = np.linalg.solve(M, rhs)
    w_np -= w_np.mean()
    with pd.Solver(omega, n, e, G) as s:
        vt = torch.from_numpy(v).cuda()
        w = pd.pairdiag_product_fit(s.h, vt, omega)
        assert np.max(np.abs(w - w_np)) < 1e-8 * max(1.0, np.max(np.abs(w_np)))
        out = torch.empty(s.dim, dtype=torch.float64, device="cuda")
        pd.pairdiag_product_start_dev(s.h, w, out)
        ex = occ @ w
        assert np.allclose(out.cpu().numpy(), np.exp(ex - ex.max()), rtol=1e-12, atol=0)
        # the fitted product vector is a good approximation of the ground state
        pv = np.exp(ex - ex.max())
        assert abs(pv @ v) / np.linalg.norm(pv) > 0.9


def test_warm_start_gain():
    """A network trained on ground states the solver computes at Omega <= 18
    starts Lanczos closer to the ground state than a random vector on held-out
    problems at Omega = 20..22: fewer iterations, the same E0."""
    train = pd_inputs.training_problems(240, seed=11, omega_lo=10, omega_hi=18)
    X, T = warmstart.training_set(train)
    ws = warmstart.WarmStart(seed=0)
    hist = ws.train(X, T, steps=2500, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    test = pd_inputs.training_problems(8, seed=99, omega_lo=20, omega_hi=22)
    it_rand, it_mlp = [], []
    for omega, n, e, G in test:
        with pd.Solver(omega, n, e, G, window=20, start=pd.PD_START_RANDOM) as s:
            r0 = s.ground_state(1e-8, want_vector=False)
        with pd.Solver(omega, n, e, G, window=20, start=pd.PD_START_MLP) as s:
            ws.attach(s.h)
            r1 = s.ground_state(1e-8, want_vector=False)
        assert r0["status"] == pd.PD_OK and r1["status"] == pd.PD_OK
        assert abs(r0["e0"] - r1["e0"]) <= 1e-9 * abs(r0["e0"])
        it_rand.append(r0["iterations"]); it_mlp.append(r1["iterations"])
    assert np.mean(it_mlp) < 0.9 * np.mean(it_rand), (it_rand, it_mlp)
    ws.close()

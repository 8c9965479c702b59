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


# ------------------------------------------------------------------------------
# Layer by layer, element by element.  Each intermediate the GPU stores is
# compared with its defining formula evaluated in FP64 on the GPU's own inputs
# to that layer (so an error is never propagated), under the rounding bound of
# the arithmetic that produced it:
#   * a tensor-core or FP32 sum of n products of bfloat16 values (exact in FP32)
#     is within gamma_n sum|terms|, gamma_n = n u / (1 - n u), taken with
#     u = 2^-23 (twice the FP32 unit roundoff, which also covers accumulation
#     that truncates instead of rounding);
#   * a value stored in bfloat16 is within 2^-8 of its magnitude (8 significant
#     bits, round to nearest);
#   * silu and silu' use a fast exp: relative 2^-14 for silu, absolute
#     2^-16 (1 + |z|) for silu'.
U_TC = 2.0 ** -23
UB16 = 2.0 ** -8


def _gam(n):
    return n * U_TC / (1.0 - n * U_TC)


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _dsilu(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


def _close(name, got, ref, bound):
    got = np.asarray(got, dtype=np.float64)
    bad = np.abs(got - ref) > bound + 1e-30
    assert not bad.any(), (name, int(bad.sum()), float(np.max(np.abs(got - ref) / (bound + 1e-30))))


@pytest.mark.parametrize("rows", [5, 64, 300, 1000, 4133])
def test_layers_element_by_element(rows):
    m, theta = _params(rows)
    W1, b1, W2, b2, W3, b3, w4, b4 = omlp.unpack(theta)
    W1, W2, W3, w4 = omlp.bf16(W1), omlp.bf16(W2), omlp.bf16(W3), omlp.bf16(w4)
    rng = np.random.default_rng(rows + 1)
    X = rng.normal(size=(rows, 16)).astype(np.float32)
    t = rng.normal(size=rows).astype(np.float32)
    loss, grad = pd.pairdiag_mlp_loss_grad(m, X, t)
    buf = lambda w: pd.pairdiag_mlp_buffer(m, w, rows).astype(np.float64)
    Xb = omlp.bf16(X)
    # forward
    A_prev = Xb
    Zs, As = [], []
    for (W, b, wz, wa) in [(W1, b1, pd.PD_MLP_Z1, pd.PD_MLP_A1), (W2, b2, pd.PD_MLP_Z2, pd.PD_MLP_A2),
                           (W3, b3, pd.PD_MLP_Z3, pd.PD_MLP_A3)]:
        Z = buf(wz)
        _close("Z", Z, A_prev @ W + b, _gam(W.shape[0] + 1) * (np.abs(A_prev) @ np.abs(W) + np.abs(b)))
        A = buf(wa)
        sz = _silu(Z)
        _close("A", A, sz, (UB16 + 2.0 ** -14) * np.abs(sz))
        Zs.append(Z); As.append(A)
        A_prev = A
    out = buf(pd.PD_MLP_OUT)
    _close("out", out, As[2] @ w4 + b4[0], _gam(129) * (np.abs(As[2]) @ np.abs(w4) + abs(b4[0])))
    # backward
    dout = buf(pd.PD_MLP_DOUT)
    d_ref = 2.0 * (out - t) / rows
    _close("dout", dout, d_ref, 3 * 2.0 ** -24 * np.abs(d_ref))
    n_grads = {}
    layers = [(3, pd.PD_MLP_DZ3, None, W3), (2, pd.PD_MLP_DZ2, pd.PD_MLP_DA2, W2), (1, pd.PD_MLP_DZ1, pd.PD_MLP_DA1, W1)]
    dZ_next = None
    for (li, wdz, wda, W) in layers:
        Z = Zs[li - 1]
        ds = _dsilu(Z)
        if li == 3:
            up = np.outer(dout, w4)                    # dA3 = dout w4^T (FP32 product per element)
            up_err = 2.0 ** -24 * np.abs(up)
        else:
            Wn = W3 if li == 2 else W2
            up = buf(wda)
            _close("dA", up, dZ_next @ Wn.T, _gam(128) * (np.abs(dZ_next) @ np.abs(Wn).T))
            up_err = 0.0
        dz_exact = up * ds
        dz_err = 2.0 ** -24 * np.abs(dz_exact) + np.abs(up) * 2.0 ** -16 * (1.0 + np.abs(Z)) + up_err * np.abs(ds)
        dZ = buf(wdz)
        _close("dZ", dZ, dz_exact, UB16 * np.abs(dz_exact) * (1 + UB16) + 2 * dz_err)
        # bias gradient: the FP32 sum of the unrounded dz over the rows
        n_grads["b%d" % li] = (dz_exact.sum(axis=0), _gam(rows) * np.abs(dz_exact).sum(axis=0) + dz_err.sum(axis=0))
        # weight gradient: the previous layer's activations against the stored dZ
        Ain = Xb if li == 1 else As[li - 2]
        n_grads["W%d" % li] = (Ain.T @ dZ, _gam(rows) * (np.abs(Ain).T @ np.abs(dZ)))
        dZ_next = dZ
    # sum of bfloat16 x FP32 products: each product rounds too (2 rows roundings)
    n_grads["w4"] = (As[2].T @ dout, _gam(2 * rows) * (np.abs(As[2]).T @ np.abs(dout)))
    n_grads["b4"] = (np.array([dout.sum()]), np.array([_gam(rows) * np.abs(dout).sum()]))
    offs = dict(W1=(0, 2048), b1=(2048, 2176), W2=(2176, 18560), b2=(18560, 18688), W3=(18688, 35072),
                b3=(35072, 35200), w4=(35200, 35328), b4=(35328, 35329))
    for name, (lo, hi) in offs.items():
        ref, bound = n_grads[name]
        _close("grad " + name, grad[lo:hi].astype(np.float64), np.ravel(ref), np.ravel(bound))
    pd.pairdiag_mlp_destroy(m)


@pytest.mark.parametrize("rows", [5, 64, 300, 1000])
def test_forward_and_gradient_vs_oracle(rows):
    """End to end, in addition to the layer checks above: the BF16 tensor-core
    forward/backward against the FP64 twin evaluated on the same
    bfloat16-rounded inputs and weights (the remaining difference is FP32
    accumulation and the bfloat16 storage of backward intermediates, which
    compound over the layers, so this comparison is per parameter group)."""
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
        # one weight per orbit of the handle, checked before the library reads w
        assert pd.pairdiag_omega(s.h) == omega
        with pytest.raises(ValueError, match=r"w must be \[12\]"):
            pd.pairdiag_product_start_dev(s.h, w[:-1], out)
        with pytest.raises(ValueError, match=r"w must be \[12\]"):
            pd.pairdiag_set_start_weights(s.h, np.r_[w, 0.0])
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

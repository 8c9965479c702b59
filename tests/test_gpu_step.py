"""The fused Lanczos step (one cooperative launch per step: the three-term
recurrence, one full Gram-Schmidt pass against the window, the norm and the
scaling into the next basis vector; Algorithm 2 with Sec. 3.4's full
reorthogonalisation) against the oracle's Lanczos and against the three-launch
form of the same step."""
import math

import numpy as np
import pytest

import oracle
import pd_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_2001_01978_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def ritz_after(omega, n, e, G, start, window, fused, precision=None):
    """Lowest Ritz value of one Krylov space of `window` steps from `start`
    (mode 1: no restart, no early stop)."""
    prec = pd.PD_PREC_FP64 if precision is None else precision
    with pd.Solver(omega, n, e, G, precision=prec, window=window, mode=1, start=pd.PD_START_USER) as s:
        pd.pairdiag_set_step_fusion(s.h, fused)
        pd.pairdiag_set_start(s.h, start)
        return s.ground_state(1e-30, want_vector=False)


# dims from one CTA to several hundred thousand states, with ragged tails
# (dim mod 4 != 0: the last pack of every vector is partial)
@pytest.mark.parametrize("omega,n,window", [(9, 4, 5), (15, 4, 12), (13, 6, 30), (17, 8, 12), (19, 7, 20),
                                            (21, 10, 9), (16, 3, 64)])
def test_krylov_space_ritz_value_vs_oracle(omega, n, window):
    """After `window` steps from the same start the lowest Ritz value of the
    fused FP64 step equals the oracle's (every alpha_i, beta_i enters it)."""
    e, G = pd_inputs.separable_noise(omega, seed=omega * 5 + n)
    dim = math.comb(omega, n)
    window = min(window, dim)
    start = pd_inputs.random_vector(dim, 100 + omega)
    ref = oracle.lanczos_ground(omega, n, e, G, start=start, window=window, tol=1e-30, mode=1)["e0"]
    r = ritz_after(omega, n, e, G, start, window, True)
    assert abs(r["e0"] - ref) <= 1e-11 * abs(ref), (r["e0"], ref)
    assert r["iterations"] == window          # no breakdown from a random start


@pytest.mark.parametrize("omega,n", [(14, 7), (20, 9), (23, 11)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_and_three_launch_forms_agree(omega, n, precision):
    """Restarted solves with the fused step and with the three-launch step:
    the same E0 to 1e-12 (FP64) or within the tolerance's energy error (mixed),
    and iteration counts within one cycle."""
    e, G = pd_inputs.separable_noise(omega, seed=omega + 17 * n)
    prec = pd.PD_PREC_FP64 if precision == "fp64" else pd.PD_PREC_MIXED
    out = []
    for fused in (True, False):
        with pd.Solver(omega, n, e, G, precision=prec, window=20, seed=3) as s:
            pd.pairdiag_set_step_fusion(s.h, fused)
            out.append(s.ground_state(1e-9, want_vector=False))
    a, b = out
    assert a["status"] == pd.PD_OK and b["status"] == pd.PD_OK
    assert abs(a["e0"] - b["e0"]) <= (1e-12 if precision == "fp64" else 1e-10) * abs(b["e0"])
    assert abs(a["iterations"] - b["iterations"]) <= 20


def test_fused_step_work_vector_in_global_memory():
    """Omega=26, N=13 (dim 1.04e7): each CTA's slice of p is too large for
    shared memory, so the fused step keeps p in global memory.  FP32 Krylov
    space of 12 steps: the same Ritz value as the three-launch form, and both
    within FP32 rounding of the FP64 one."""
    omega, n = 26, 13
    e, G = pd_inputs.separable_noise(omega, seed=29)
    dim = math.comb(omega, n)
    start = pd_inputs.random_vector(dim, 7)
    f32 = [ritz_after(omega, n, e, G, start, 12, fused, pd.PD_PREC_MIXED)["e0"] for fused in (True, False)]
    f64 = ritz_after(omega, n, e, G, start, 12, True)["e0"]
    assert abs(f32[0] - f32[1]) <= 1e-6 * abs(f64)
    assert abs(f32[0] - f64) <= 1e-5 * abs(f64)

"""Batched ground states (many Hamiltonians in one run) against the CPU oracle
and against single-problem solves."""
import math

import numpy as np
import pytest

import oracle
import pd_inputs
from conftest import read_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_2001_01978_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    yield
    torch.cuda.synchronize()


def small_batch():
    probs = []
    spec = [(6, 3), (7, 0), (8, 1), (9, 8), (10, 5), (11, 4), (12, 6), (13, 7), (14, 5), (15, 9), (16, 8), (17, 6)]
    for i, (om, n) in enumerate(spec):
        e, G = pd_inputs.separable_noise(om, seed=100 + i)
        probs.append((om, n, e, G))
    return probs


@pytest.mark.parametrize("precision,rel", [(0, 1e-11), (1, 1e-8)])
def test_small_batch_vs_oracle(precision, rel):
    probs = small_batch()
    opt = pd.pairdiag_default_options(precision=precision, window=20)
    r = pd.pairdiag_batch_ground_state(probs, 1e-11 if precision == 0 else 1e-6, opt)
    assert r["call_status"] == pd.PD_OK, r["status"]
    for i, (om, n, e, G) in enumerate(probs):
        ref = oracle.lanczos_ground(om, n, e, G, window=40, tol=1e-13)["e0"]
        scale = max(1.0, abs(ref))
        assert abs(r["e0"][i] - ref) <= rel * scale, (i, om, n, r["e0"][i], ref)
        assert r["converged"][i] == 1
    assert np.all(r["latency_ms"] > 0) or r["latency_ms"].max() > 0


def test_batch_matches_single_solves_fp64():
    probs = small_batch()
    opt = pd.pairdiag_default_options(precision=pd.PD_PREC_FP64, window=20, seed=7)
    r = pd.pairdiag_batch_ground_state(probs, 1e-12, opt)
    for i, (om, n, e, G) in enumerate(probs):
        with pd.Solver(om, n, e, G, window=20, seed=7) as s:
            one = s.ground_state(1e-12, want_vector=False)
        assert abs(r["e0"][i] - one["e0"]) <= 1e-11 * max(1.0, abs(one["e0"]))


def test_workload_4096_stratified_subset():
    """The 4096-problem mean-field workload (Omega ~ U{10..22}): mixed form in one
    run, every problem converged; twelve stratified picks against the oracle's
    E0 -- computed here for dim <= 20000, read from the values that
    tests/golden/make_golden.py wrote with the oracle for the larger ones."""
    probs = pd_inputs.batch_workload(4096, seed=5)
    opt = pd.pairdiag_default_options(precision=pd.PD_PREC_MIXED, window=20)
    r = pd.pairdiag_batch_ground_state(probs, 1e-6, opt)
    assert r["call_status"] == pd.PD_OK
    assert np.all(r["converged"] == 1), np.flatnonzero(r["converged"] != 1)[:10]
    dims = np.array([math.comb(om, n) for om, n, _, _ in probs])
    order = np.argsort(dims, kind="stable")
    picks = [int(order[k]) for k in np.linspace(0, len(order) - 1, 12).astype(int)]
    golden = {int(row[0]): (int(row[1]), int(row[2]), float(row[4]))
              for row in read_golden("batch4096_s5_picks_e0.txt")}
    assert sorted(golden) == sorted(picks)
    for i in picks:
        om, n, e, G = probs[i]
        if dims[i] <= 20000:
            ref = oracle.lanczos_ground(om, n, e, G, window=40, tol=1e-12)["e0"]
        else:
            assert golden[i][:2] == (om, n)
            ref = golden[i][2]
        assert abs(r["e0"][i] - ref) <= 1e-8 * max(1.0, abs(ref)), (i, om, n, dims[i], r["e0"][i], ref)


def test_batch_on_reused_device_blocks():
    """A batch call that receives the device blocks an earlier call left in the
    library's cache (old data in them) gives the oracle's energies, and every
    problem smaller than the window finishes within dim + 2 Lanczos steps, as
    a Krylov space that spans it must (a skipped alpha dot stalls them)."""
    probs = small_batch()
    pd.pairdiag_batch_ground_state(probs, 1e-11, pd.pairdiag_default_options(precision=0, window=20))
    r = pd.pairdiag_batch_ground_state(probs, 1e-6, pd.pairdiag_default_options(precision=1, window=20))
    assert r["call_status"] == pd.PD_OK
    for i, (om, n, e, G) in enumerate(probs):
        ref = oracle.lanczos_ground(om, n, e, G, window=40, tol=1e-13)["e0"]
        assert abs(r["e0"][i] - ref) <= 1e-8 * max(1.0, abs(ref)), (i, r["e0"][i], ref)
        dim = math.comb(om, n)
        if dim < 20:
            assert r["iterations"][i] <= dim + 2, (i, dim, r["iterations"][i])

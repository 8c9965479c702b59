"""The seeded input generators shared by both sides (CPU only)."""
import math

import numpy as np

import pd_inputs


def test_splitmix64_published_sequence():
    """SplitMix64 from state 0 (Steele, Lea & Flood): the first three outputs."""
    got = [int(v) for v in pd_inputs.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # counters are positions: an offset continues the same sequence
    assert int(pd_inputs.splitmix64(0, 1, offset=2)[0]) == got[2]
    u = pd_inputs.splitmix_uniform(7, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01


def test_separable_and_constant_noise_shapes():
    for omega, seed in ((24, 1), (30, 2)):
        e, G = pd_inputs.separable_noise(omega, seed)
        assert e.shape == (omega,) and G.shape == (omega, omega)
        assert np.array_equal(G, G.T) and np.all(np.diff(e) >= 0)
        assert np.all(np.abs(e) <= 10.0)
        e2, G2 = pd_inputs.separable_noise(omega, seed)
        assert np.array_equal(e, e2) and np.array_equal(G, G2)
    e, G = pd_inputs.constant_noise(32, 3)
    assert np.array_equal(G, G.T) and abs(G.mean() + 0.4) < 0.02


def test_batch_workload_recipe():
    probs = pd_inputs.batch_workload()
    assert len(probs) == 4096
    dims = []
    for omega, n, e, G in probs:
        assert 10 <= omega <= 22 and 1 <= n <= omega - 1
        assert abs(n - omega // 2) <= 3
        assert np.array_equal(G, G.T) and e.shape == (omega,)
        dims.append(math.comb(omega, n))
    assert max(dims) <= math.comb(22, 11)
    assert 5e4 < np.mean(dims) < 1.5e5
    # a few positive entries come from the noise on small products g_i g_j
    pos = np.mean([np.mean(G > 0) for _, _, _, G in probs[:200]])
    assert 0.0 <= pos < 0.01

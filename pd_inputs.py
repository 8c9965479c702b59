"""Seeded synthetic inputs for the pairing-Hamiltonian workloads.

This module is shared by the CPU oracle's tests and by the CUDA path's tests and
benchmark.  It holds no arithmetic of the method itself (no basis, no ranking, no
Hamiltonian): only the draws of single-particle energies e_i and pairing
strengths G_ij, start/test vectors, and the counter-based generator that both
sides implement from its published definition.

Conventions (Eq. 2 of the paper, pair form): H = sum_i (2 e_i + G_ii) n_i
+ sum_{i != j} G_ij P_i^+ P_j, with G real symmetric, orbit 0 = bit 0.

Draw order for the seeded configurations (numpy ``default_rng(seed)``, PCG64):
  1. e (Omega uniform draws; sorted where the workload says so),
  2. g (Omega uniform draws in [0.3, 0.7]) for the separable-plus-noise form,
  3. eta: the upper triangle including the diagonal, row-major, N(0, sigma^2),
     mirrored to the lower triangle.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# Paper-style workloads (Section 5: e_i = 1..Omega, constant G)
# ---------------------------------------------------------------------------
def picket_fence(omega: int, g: float, first: float = 1.0, g_float32: bool = False):
    """e_i = first, first+1, ...; G_ij = g for all i, j.

    ``g_float32`` rounds g to IEEE single precision first: the Fortran default-REAL
    literal of the paper's example program (Appendix A) behaves this way, and the
    digits printed in Tables 2 and 3 follow that rounding.
    """
    gv = float(np.float32(g)) if g_float32 else float(g)
    e = first + np.arange(omega, dtype=np.float64)
    G = np.full((omega, omega), gv, dtype=np.float64)
    return e, G


def _sym_noise(rng, omega: int, sigma: float) -> np.ndarray:
    eta = np.zeros((omega, omega))
    iu = np.triu_indices(omega)
    eta[iu] = rng.normal(0.0, sigma, size=len(iu[0]))
    return eta + np.triu(eta, 1).T


def separable_noise(omega: int, seed: int, sort_e: bool = True, sigma: float = 0.05):
    """e ~ U[-10,10] (sorted), G_ij = -g_i g_j + eta_ij, g ~ U[0.3,0.7], eta ~ N(0, sigma^2) symmetric."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-10.0, 10.0, size=omega)
    if sort_e:
        e = np.sort(e)
    g = rng.uniform(0.3, 0.7, size=omega)
    G = -np.outer(g, g) + _sym_noise(rng, omega, sigma)
    return e, G


def constant_noise(omega: int, seed: int, g0: float = -0.4, sigma: float = 0.05):
    """e ~ U[-10,10] (unsorted), G_ij = g0 + eta_ij with symmetric Gaussian eta."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-10.0, 10.0, size=omega)
    G = g0 + _sym_noise(rng, omega, sigma)
    return e, G


# ---------------------------------------------------------------------------
# The named workloads
# ---------------------------------------------------------------------------
WORKLOADS = {
    "omega12_n6_picket": dict(omega=12, n_pairs=6),
    "omega24_n12_sepnoise_s1": dict(omega=24, n_pairs=12),
    "omega30_n15_sepnoise_s2": dict(omega=30, n_pairs=15),
    "omega32_n16_constnoise_s3": dict(omega=32, n_pairs=16),
}


def workload(name: str):
    """Return (omega, n_pairs, e, G) for a named workload."""
    if name == "omega12_n6_picket":
        # e_i = i for i = 0..11, G = -0.5 everywhere.
        e, G = picket_fence(12, -0.5, first=0.0)
        return 12, 6, e, G
    if name == "omega24_n12_sepnoise_s1":
        e, G = separable_noise(24, seed=1)
        return 24, 12, e, G
    if name == "omega30_n15_sepnoise_s2":
        e, G = separable_noise(30, seed=2)
        return 30, 15, e, G
    if name == "omega32_n16_constnoise_s3":
        e, G = constant_noise(32, seed=3)
        return 32, 16, e, G
    raise KeyError(name)


def batch_workload(count: int = 4096, seed: int = 5, omega_lo: int = 10, omega_hi: int = 22):
    """Mean-field-style batch: Omega ~ U{lo..hi}, N = floor(Omega/2) + s*u with
    s in {-1,+1}, u ~ U{0..3}, clamped to [1, Omega-1]; e ~ U[-10,10];
    G = -g g^T + eta as in the separable workload.  Draws per problem, in order:
    Omega, s, u, e, g, eta."""
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(count):
        omega = int(rng.integers(omega_lo, omega_hi + 1))
        s = 1 if int(rng.integers(0, 2)) else -1
        u = int(rng.integers(0, 4))
        n = min(max(omega // 2 + s * u, 1), omega - 1)
        e = rng.uniform(-10.0, 10.0, size=omega)
        g = rng.uniform(0.3, 0.7, size=omega)
        G = -np.outer(g, g) + _sym_noise(rng, omega, 0.05)
        probs.append((omega, n, e, G))
    return probs


def training_problems(count: int, seed: int, omega_lo: int = 10, omega_hi: int = 18):
    """Problems for training the warm-start network: the mean-field batch
    distribution restricted to Omega in [omega_lo, omega_hi], plus picket-fence
    spectra with constant G drawn in [-1, -0.1] for every fifth problem."""
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(count):
        omega = int(rng.integers(omega_lo, omega_hi + 1))
        n = min(max(omega // 2 + int(rng.integers(-3, 4)), 1), omega - 1)
        if i % 5 == 4:
            e = np.arange(omega, dtype=np.float64) * float(rng.uniform(0.5, 2.0))
            G = np.full((omega, omega), float(rng.uniform(-1.0, -0.1)))
        else:
            e = rng.uniform(-10.0, 10.0, size=omega)
            g = rng.uniform(0.3, 0.7, size=omega)
            G = -np.outer(g, g) + _sym_noise(rng, omega, 0.05)
        probs.append((omega, n, e, G))
    return probs


def n_states(omega: int, n: int) -> int:
    """Number of pair configurations, for sizing buffers (math.comb)."""
    return math.comb(omega, n) if 0 <= n <= omega else 0


# ---------------------------------------------------------------------------
# Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the value at
# counter i is the SplitMix64 output mix applied to seed + (i + 1) * gamma.
# Both the CPU and the CUDA side implement this definition; it fixes the
# seeded random Lanczos start vector.
# ---------------------------------------------------------------------------
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """uint64 outputs for counters offset .. offset+count-1."""
    with np.errstate(over="ignore"):
        i = np.arange(offset, offset + count, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + (i + np.uint64(1)) * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def splitmix_uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [-1, 1): top 53 bits of each output scaled to [0,1), then 2u-1."""
    z = splitmix64(seed, count, offset)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def random_vector(n: int, seed: int) -> np.ndarray:
    """A plain N(0,1) test vector (numpy PCG64)."""
    return np.random.default_rng(seed).standard_normal(n)

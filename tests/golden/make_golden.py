"""Write oracle-computed expected values for workloads too large to solve
inside the test-suite.  Calls only ``oracle/`` (and the seeded inputs).

    python tests/golden/make_golden.py omega24_n12_sepnoise_s1
    python tests/golden/make_golden.py odd:25:12:1:11     # Omega, pairs, seed, blocked orbit
    python tests/golden/make_golden.py batch:4096:5       # problem count, seed
"""
import sys
import time
from pathlib import Path

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parent.parent))

import oracle  # noqa: E402
import pd_inputs  # noqa: E402


def ground_state(name: str, window: int = 50, tol: float = 1e-12):
    omega, n, e, G = pd_inputs.workload(name)
    t0 = time.time()
    r = oracle.lanczos_ground(omega, n, e, G, window=window, tol=tol, max_restarts=400)
    dt = time.time() - t0
    out = HERE / f"{name}_e0.txt"
    out.write_text(
        "# Oracle restarted Lanczos (Algorithm 2, full reorthogonalisation, e_1 start),\n"
        f"# window {window}, |beta_1/alpha_1| <= {tol:g}; written by tests/golden/make_golden.py.\n"
        "# Columns: E0 rel_residual iterations restarts converged gap_estimate seconds\n"
        f"{r['e0']!r} {r['rel_residual']!r} {r['iterations']} {r['restarts']} {int(r['converged'])} "
        f"{r['gap']!r} {dt:.1f}\n")
    print(out.read_text())


def odd_subspace(omega: int, n: int, seed: int, block: int, window: int = 50, tol: float = 1e-12):
    """E_b of one blocked subspace (Eq. 3) of the separable workload with `seed`."""
    from oracle import odd
    e, G = pd_inputs.separable_noise(omega, seed=seed)
    t0 = time.time()
    r = odd.blocked_ground(omega, n, e, G, block=block, tol=tol, window=window, max_restarts=400)
    dt = time.time() - t0
    out = HERE / f"omega{omega}_n{n}_sepnoise_s{seed}_odd_b{block}_e0.txt"
    out.write_text(
        f"# Odd mass (Eq. 3): {omega} orbits, {n} pairs + 1 particle blocking orbit {block} (0-based);\n"
        "# e, G = pd_inputs.separable_noise(omega, seed).  Oracle restarted Lanczos on the other\n"
        f"# orbits, window {window}, |beta_1/alpha_1| <= {tol:g}; written by tests/golden/make_golden.py.\n"
        "# Columns: E_b converged seconds\n"
        f"{r['e0']!r} {int(r['converged'])} {dt:.1f}\n")
    print(out.read_text())


def batch_picks(count: int, seed: int):
    """Stratified picks of the mean-field batch workload (12 problems at evenly
    spaced ranks of the dimension) and the oracle's E0 of each: the benchmark
    reports the batch's error against them, and the test-suite reads the picks
    it cannot afford to solve itself (dim > 20000)."""
    import math

    import numpy as np
    probs = pd_inputs.batch_workload(count, seed=seed)
    dims = np.array([math.comb(om, n) for om, n, _, _ in probs])
    order = np.argsort(dims, kind="stable")
    picks = [int(order[k]) for k in np.linspace(0, len(order) - 1, 12).astype(int)]
    lines = []
    for i in picks:
        om, n, e, G = probs[i]
        t0 = time.time()
        r = oracle.lanczos_ground(om, n, e, G, window=50, tol=1e-12, max_restarts=400)
        dt = time.time() - t0
        lines.append(f"{i} {om} {n} {dims[i]} {r['e0']!r} {r['rel_residual']!r} {int(r['converged'])} {dt:.1f}")
        print(lines[-1], flush=True)
    out = HERE / f"batch{count}_s{seed}_picks_e0.txt"
    out.write_text(
        f"# Mean-field batch workload: pd_inputs.batch_workload({count}, seed={seed}); stratified picks\n"
        "# (12 evenly spaced ranks of dim, stable argsort).  Oracle restarted\n"
        "# Lanczos (Algorithm 2, full reorthogonalisation, e_1 start), window 50, |beta_1/alpha_1| <= 1e-12;\n"
        "# written by tests/golden/make_golden.py.\n"
        "# Columns: problem omega n_pairs dim E0 rel_residual converged seconds\n" + "\n".join(lines) + "\n")
    print(out.read_text())


if __name__ == "__main__":
    for name in sys.argv[1:]:
        if name.startswith("batch:"):
            count, seed = (int(v) for v in name.split(":")[1:])
            batch_picks(count, seed)
        elif name.startswith("odd:"):
            omega, n, seed, block = (int(v) for v in name.split(":")[1:])
            odd_subspace(omega, n, seed, block)
        else:
            ground_state(name)

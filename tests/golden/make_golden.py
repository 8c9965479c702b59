"""Write oracle-computed expected values for workloads too large to solve
inside the test-suite.  Calls only ``oracle/`` (and the seeded inputs).

    python tests/golden/make_golden.py omega24_n12_sepnoise_s1
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


if __name__ == "__main__":
    for name in sys.argv[1:]:
        ground_state(name)

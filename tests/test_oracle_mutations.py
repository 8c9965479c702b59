"""Plant plausible mistakes in a copy of the oracle's C source and check that
the paper pins catch each one (CPU only; the planted copies live in a temp dir)."""
import ctypes
import subprocess
from pathlib import Path

import numpy as np
import pytest

import oracle
import pd_inputs
from conftest import read_golden

SRC = Path(oracle.__file__).resolve().parent / "pd_oracle.c"

MUTATIONS = {
    "diag_drops_self_energy": ("2.0 * e[p] + G[p * omega + p]", "2.0 * e[p]"),
    "diag_single_e": ("2.0 * e[p] + G[p * omega + p]", "e[p] + G[p * omega + p]"),
    "hash_wrong_orbit_offset": ("f += orc_binom(O - 1, j);", "f += orc_binom(O, j);"),
    "successor_no_refill": ("for (int i = 0; i < j; ++i) c[i] = i;", "for (int i = 0; i < j; ++i) c[i] = c[i];"),
    "offdiag_wrong_sign": ("acc += G[q * omega + o] * x[j];", "acc -= G[q * omega + o] * x[j];"),
    "jacobi_wrong_rotation_sign": ("A[k * n + p] = c * akp - s * akq;", "A[k * n + p] = c * akp + s * akq;"),
}


def _build(tmp_path, name, old, new):
    text = SRC.read_text()
    assert old in text, name
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", str(src), "-o", str(so), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    P, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    L.orc_build_basis.restype = i64; L.orc_build_basis.argtypes = [i32, i32, P]
    L.orc_hash.restype = u64; L.orc_hash.argtypes = [u64]
    L.orc_hx.restype = None; L.orc_hx.argtypes = [i32, P, P, P, i64, P, P]
    L.orc_jacobi.restype = None; L.orc_jacobi.argtypes = [i32, P, P, P]
    return L


def _pins_hold(L) -> bool:
    """Table 1, the hash examples, the worked 6x6 matrix and a Jacobi check."""
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    b = np.zeros(6, dtype=np.uint64)
    if L.orc_build_basis(4, 2, p(b)) != 6 or list(b) != [3, 5, 6, 9, 10, 12]:
        return False
    for bits, f in read_golden("hash_examples.txt"):
        if L.orc_hash(int(bits, 2)) != int(f):
            return False
    M = np.array([[float(v) for v in r] for r in read_golden("matrix_4_2_g02.txt")])
    e, G = pd_inputs.picket_fence(4, -0.2)
    for j in range(6):
        x = np.zeros(6); x[j] = 1.0; y = np.zeros(6)
        L.orc_hx(4, p(e), p(G), p(b), 6, p(x), p(y))
        if not np.allclose(y, M[:, j], atol=1e-14):
            return False
    A = np.array([[2.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 4.0]])
    w = np.zeros(3); V = np.zeros((3, 3)); Ac = A.copy()
    L.orc_jacobi(3, p(Ac), p(w), p(V))
    return bool(np.allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-12))


def test_unmutated_copy_passes(tmp_path):
    assert _pins_hold(_build(tmp_path, "clean", "/*", "/*"))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    assert not _pins_hold(_build(tmp_path, name, old, new))

"""CPU FP64 oracle for the pairing-Hamiltonian ground state (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2001_01978_gb300``) and neither imports the other.

Contents
  * ``pd_oracle.c`` (loaded through ctypes): binomials (Eq. extcmn), the
    successor of k-subsets in colexicographic order (Knuth's Algorithm L), the
    basis in the order of Sec. 3.1, binary search and
    the hash (Sec. 3.2), the diagonal element (Eq. diagonal), H*x by explicit
    scattering (Sec. 3.3), restarted Lanczos with full reorthogonalisation
    (Algorithm 2, Sec. 3.4), cyclic Jacobi.
  * ``richardson.py``: the constant-G ground-state energy from Richardson's
    equations in their eigenvalue-based form (an independent route, used as a
    pin for the matrix path).
  * ``mlp.py``: the FP64 twin of the warm-start network (forward/backward).
  * ``odd.py``: odd-mass systems in the blocking approximation (Eq. 3): every
    blocked subspace solved as a seniority-zero problem on the other orbits.
  * ``excited.py``: the lowest few eigenpairs (Sec. 3.4) of small problems from
    the dense matrix.
  * ``truncation.py``: the truncated space of Sec. 3.5 (histogram cutoff of the
    diagonal elements) and H*x on it by binary search.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against the
paper's printed values, closed forms, invariants or brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pd_oracle.c"
_LIB = _HERE / "_build" / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile pd_oracle.c into oracle/_build/liboracle.so with gcc (-O2, OpenMP,
    no floating-point contraction so that both host architectures round alike)."""
    _LIB.parent.mkdir(parents=True, exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(".so.tmp%d" % os.getpid())
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", str(_SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        u64, i64, i32, dbl = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        P = ctypes.c_void_p
        L.orc_binom.restype = u64; L.orc_binom.argtypes = [i32, i32]
        L.orc_next_state.restype = u64; L.orc_next_state.argtypes = [u64]
        L.orc_build_basis.restype = i64; L.orc_build_basis.argtypes = [i32, i32, P]
        L.orc_search.restype = i64; L.orc_search.argtypes = [P, i64, u64]
        L.orc_hash.restype = u64; L.orc_hash.argtypes = [u64]
        L.orc_diag.restype = dbl; L.orc_diag.argtypes = [u64, i32, P, P]
        L.orc_hx.restype = None; L.orc_hx.argtypes = [i32, P, P, P, i64, P, P]
        L.orc_hx_rows.restype = None; L.orc_hx_rows.argtypes = [i32, P, P, P, i64, P, P, i64, P]
        L.orc_hx_sub.restype = None; L.orc_hx_sub.argtypes = [i32, P, P, P, i64, P, P]
        L.orc_monopole.restype = None; L.orc_monopole.argtypes = [i32, P, P, P, i64, P, P, P]
        L.orc_jacobi.restype = None; L.orc_jacobi.argtypes = [i32, P, P, P]
        L.orc_lanczos_ground.restype = i32
        L.orc_lanczos_ground.argtypes = [i32, i32, P, P, i32, dbl, i32, i32, P, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def binom(n: int, m: int) -> int:
    """Eq. (extcmn), extended to 0 for n < m."""
    return int(lib().orc_binom(n, m))


def next_state(s: int) -> int:
    """Next larger word with the same popcount (the order of Sec. 3.1), by the
    textbook successor of k-subsets in colexicographic order (Knuth, TAOCP 4A,
    Sec. 7.2.1.3, Algorithm L)."""
    return int(lib().orc_next_state(s))


def basis(omega: int, n: int) -> np.ndarray:
    """Ascending basis of all omega-bit words with n set bits (Sec. 3.1, Table 1)."""
    dim = binom(omega, n)
    out = np.zeros(dim, dtype=np.uint64)
    got = lib().orc_build_basis(omega, n, _p(out))
    assert got == dim, (got, dim)
    return out


def search(b: np.ndarray, s: int) -> int:
    """Binary search (Sec. 3.2); -1 when absent."""
    b = np.ascontiguousarray(b, dtype=np.uint64)
    return int(lib().orc_search(_p(b), len(b), s))


def hash_index(s: int) -> int:
    """The paper's 1-based hash f(s) (Sec. 3.2)."""
    return int(lib().orc_hash(s))


def diag(s: int, e, G) -> float:
    e = _f64(e); G = _f64(G)
    return float(lib().orc_diag(s, len(e), _p(e), _p(G)))


def hx(omega: int, n: int, e, G, x, b: np.ndarray | None = None) -> np.ndarray:
    """y = H x by explicit scattering with binary search (Sec. 3.3)."""
    e = _f64(e); G = _f64(G); x = _f64(x)
    if b is None:
        b = basis(omega, n)
    y = np.empty(len(b))
    lib().orc_hx(omega, _p(e), _p(G), _p(b), len(b), _p(x), _p(y))
    return y


def hx_rows(omega: int, n: int, e, G, x, rows, b: np.ndarray | None = None) -> np.ndarray:
    """(H x)[rows] only; for sampled checks at sizes too large for a full product."""
    e = _f64(e); G = _f64(G); x = _f64(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if b is None:
        b = basis(omega, n)
    y = np.empty(len(rows))
    lib().orc_hx_rows(omega, _p(e), _p(G), _p(b), len(b), _p(x), _p(rows), len(rows), _p(y))
    return y


def monopole(omega: int, n: int, e, G, b: np.ndarray | None = None):
    """(Monopole_Min, Monopole_Max, Posit_Min): extreme diagonal elements."""
    e = _f64(e); G = _f64(G)
    if b is None:
        b = basis(omega, n)
    lo = np.zeros(1); hi = np.zeros(1); pos = np.zeros(1, dtype=np.int64)
    lib().orc_monopole(omega, _p(e), _p(G), _p(b), len(b), _p(lo), _p(hi), _p(pos))
    return float(lo[0]), float(hi[0]), int(pos[0])


def jacobi(A) -> tuple[np.ndarray, np.ndarray]:
    """Cyclic Jacobi eigen-decomposition of a dense symmetric matrix."""
    A = np.array(A, dtype=np.float64, copy=True, order="C")
    n = A.shape[0]
    w = np.empty(n); V = np.empty((n, n))
    lib().orc_jacobi(n, _p(A), _p(w), _p(V))
    return w, V


def dense_matrix(omega: int, n: int, e, G) -> np.ndarray:
    """The full matrix, column by column, as H applied to unit vectors."""
    b = basis(omega, n)
    dim = len(b)
    M = np.empty((dim, dim))
    x = np.zeros(dim)
    for j in range(dim):
        x[:] = 0.0; x[j] = 1.0
        M[:, j] = hx(omega, n, e, G, x, b)
    return M


def lanczos_ground(omega: int, n: int, e, G, start=None, window: int = 50, tol: float = 1e-12,
                   max_restarts: int = 500, mode: int = 0) -> dict:
    """Restarted Lanczos (Algorithm 2 + Sec. 3.4).  ``start`` defaults to the
    paper's [1, 0, ..., 0]."""
    e = _f64(e); G = _f64(G)
    dim = binom(omega, n)
    if start is None:
        v = np.zeros(dim); v[0] = 1.0
    else:
        v = _f64(start).copy()
    e0 = np.zeros(1); it = np.zeros(1, dtype=np.int32); rs = np.zeros(1, dtype=np.int32)
    rel = np.zeros(1); gap = np.zeros(1)
    st = lib().orc_lanczos_ground(omega, n, _p(e), _p(G), window, tol, max_restarts, mode,
                                  _p(v), _p(e0), _p(it), _p(rs), _p(rel), _p(gap))
    if st < 0:
        raise ValueError("bad input")
    return dict(e0=float(e0[0]), vec=v, iterations=int(it[0]), restarts=int(rs[0]),
                rel_residual=float(rel[0]), gap=float(gap[0]), converged=(st == 0))

"""Thin ctypes binding of libpairdiag (include/pairdiag.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch CUDA tensors (PyTorch supplies device memory
and streams); host buffers are numpy arrays.  If the library is missing, the
import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

from . import build as _build

PD_OK, PD_EINVAL, PD_ENOMEM, PD_ENOCONV, PD_ETIMEOUT, PD_ECUDA, PD_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
PD_PREC_FP64, PD_PREC_MIXED = 0, 1
PD_HX_FLOATFLOAT = 2     # pairdiag_hx_dev only: float x, double y, float-float rows
PD_START_RANDOM, PD_START_FIRST, PD_START_HF, PD_START_USER, PD_START_MLP = 0, 1, 2, 3, 4
(PD_MLP_Z1, PD_MLP_A1, PD_MLP_Z2, PD_MLP_A2, PD_MLP_Z3, PD_MLP_A3, PD_MLP_OUT, PD_MLP_DOUT, PD_MLP_DZ3, PD_MLP_DA2,
 PD_MLP_DZ2, PD_MLP_DA1, PD_MLP_DZ1) = range(13)


class pairdiag_options(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("max_restarts", ctypes.c_int), ("precision", ctypes.c_int),
                ("start", ctypes.c_int), ("seed", ctypes.c_uint64), ("mode", ctypes.c_int),
                ("low_bits", ctypes.c_int), ("mixed_floor", ctypes.c_double), ("hx_variant", ctypes.c_int)]


class pairdiag_info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int64), ("nnz_offdiag", ctypes.c_int64), ("iterations", ctypes.c_int),
                ("hx_products", ctypes.c_int), ("iterations_fp32", ctypes.c_int), ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("gap_estimate", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class pairdiag_batch_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("stalled", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class pairdiag_tune_entry(ctypes.Structure):
    _fields_ = [("low_bits", ctypes.c_int), ("hx_variant", ctypes.c_int), ("ms", ctypes.c_double)]


class PairDiagError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_P = ctypes.c_void_p
_H = ctypes.c_void_p
_lib = None

_SIGNATURES = {
    "pairdiag_default_options": (None, [ctypes.POINTER(pairdiag_options)]),
    "pairdiag_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pairdiag_last_error": (ctypes.c_char_p, []),
    "pairdiag_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.POINTER(pairdiag_options),
                                       ctypes.POINTER(_H)]),
    "pairdiag_destroy": (None, [_H]),
    "pairdiag_set_stream": (ctypes.c_int, [_H, _P]),
    "pairdiag_dim": (ctypes.c_int64, [_H]),
    "pairdiag_nnz": (ctypes.c_int64, [_H]),
    "pairdiag_omega": (ctypes.c_int, [_H]),
    "pairdiag_basis_dev": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_int64, _P]),
    "pairdiag_basis": (ctypes.c_int, [_H, _P]),
    "pairdiag_rank_dev": (ctypes.c_int, [_H, _P, ctypes.c_int64, _P]),
    "pairdiag_hx_dev": (ctypes.c_int, [_H, ctypes.c_int, _P, _P]),
    "pairdiag_hx": (ctypes.c_int, [_H, _P, _P]),
    "pairdiag_monopole": (ctypes.c_int, [_H, _P, _P, _P]),
    "pairdiag_set_start": (ctypes.c_int, [_H, _P]),
    "pairdiag_ground_state": (ctypes.c_int, [_H, ctypes.c_double, _P, _P, ctypes.POINTER(pairdiag_info)]),
    "pairdiag_ground_state_dev": (ctypes.c_int, [_H, ctypes.c_double, _P, _P, ctypes.POINTER(pairdiag_info)]),
    "pairdiag_occupations_dev": (ctypes.c_int, [_H, _P, _P]),
    "pairdiag_lowest_states_dev": (ctypes.c_int, [_H, ctypes.c_int, ctypes.c_double, _P, _P,
                                                  ctypes.POINTER(pairdiag_info)]),
    "pairdiag_mlp_buffer": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "pairdiag_truncate": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "pairdiag_kept_map_dev": (ctypes.c_int, [_H, _P]),
    "pairdiag_full_dim": (ctypes.c_int64, [_H]),
    "pairdiag_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    "pairdiag_multidot": (ctypes.c_int, [_H, ctypes.c_int, _P, ctypes.c_int64, ctypes.c_int, _P, ctypes.c_int64, _P]),
    "pairdiag_tridiag_lowest": (ctypes.c_int, [_H, ctypes.c_int, _P, _P, _P, _P]),
    "pairdiag_kernel_launches": (ctypes.c_int64, []),
    "pairdiag_release_cache": (ctypes.c_int, [_P]),
    "pairdiag_set_profiling": (ctypes.c_int, [_H, ctypes.c_int]),
    "pairdiag_set_step_fusion": (ctypes.c_int, [_H, ctypes.c_int]),
    "pairdiag_get_profile": (ctypes.c_int, [_H, ctypes.c_int, _P, _P]),
    "pairdiag_batch_ground_state": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, ctypes.c_double,
                                                   ctypes.POINTER(pairdiag_options), _H, _P, _P, _P, _P]),
    "pairdiag_odd_ground_state": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_double,
                                                 ctypes.POINTER(pairdiag_options), _H, _P, _P, _P, _P, _P,
                                                 ctypes.POINTER(pairdiag_info)]),
    "pairdiag_mlp_create": (ctypes.c_int, [ctypes.c_uint64, ctypes.POINTER(_H)]),
    "pairdiag_mlp_destroy": (None, [_H]),
    "pairdiag_mlp_num_params": (ctypes.c_int, []),
    "pairdiag_mlp_get_params": (ctypes.c_int, [_H, _P]),
    "pairdiag_mlp_set_params": (ctypes.c_int, [_H, _P]),
    "pairdiag_mlp_features": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "pairdiag_mlp_forward": (ctypes.c_int, [_H, ctypes.c_int, _P, _P]),
    "pairdiag_mlp_loss_grad": (ctypes.c_int, [_H, ctypes.c_int, _P, _P, _P, _P]),
    "pairdiag_mlp_train": (ctypes.c_int, [_H, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_double, _P]),
    "pairdiag_set_mlp": (ctypes.c_int, [_H, _H]),
    "pairdiag_set_start_weights": (ctypes.c_int, [_H, _P]),
    "pairdiag_product_fit": (ctypes.c_int, [_H, _P, _P]),
    "pairdiag_product_start_dev": (ctypes.c_int, [_H, _P, _P]),
    "pairdiag_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(pairdiag_tune_entry), _P, _P]),
    "pairdiag_tune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pairdiag_tune_get": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
    "pairdiag_multidot_noalloc": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int64, ctypes.c_int, _P,
                                                 ctypes.c_int64, _P, _P]),
}


def library_path() -> Path:
    return _build.LIB


def lib():
    """Load libpairdiag.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        path = library_path()
        if not path.exists():
            raise ImportError(f"libpairdiag.so not built at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(str(path))
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def _check(code: int, allow=(PD_OK,)) -> int:
    if code not in allow:
        raise PairDiagError(code, lib().pairdiag_last_error().decode())
    return code


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dev_ptr(t, dtype=None):
    """data_ptr() of a contiguous CUDA tensor (marshalling check only)."""
    if not getattr(t, "is_cuda", False):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ ABI ----
def pairdiag_default_options(**overrides) -> pairdiag_options:
    o = pairdiag_options()
    lib().pairdiag_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def pairdiag_strerror(code: int) -> str:
    return lib().pairdiag_strerror(code).decode()


def pairdiag_create(omega: int, n_pairs: int, e, G, opt: pairdiag_options | None = None):
    e = np.ascontiguousarray(e, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    if e.shape != (omega,) or G.shape != (omega, omega):
        raise ValueError("e must be [omega] and G [omega, omega]")
    h = _H()
    _check(lib().pairdiag_create(omega, n_pairs, _np_ptr(e), _np_ptr(G),
                                 ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h


def pairdiag_destroy(h) -> None:
    lib().pairdiag_destroy(h)


def pairdiag_set_stream(h, stream) -> None:
    ptr = getattr(stream, "cuda_stream", stream)
    _check(lib().pairdiag_set_stream(h, ctypes.c_void_p(int(ptr))))


def pairdiag_dim(h) -> int:
    return int(lib().pairdiag_dim(h))


def pairdiag_omega(h) -> int:
    return int(lib().pairdiag_omega(h))


def pairdiag_nnz(h) -> int:
    return int(lib().pairdiag_nnz(h))


def pairdiag_full_dim(h) -> int:
    return int(lib().pairdiag_full_dim(h))


def pairdiag_truncate(h, dimension_limit: int, bins: int = 0) -> int:
    """Truncated model space of Sec. 3.5 (0 restores the full space); returns the
    new dimension (the kept states)."""
    kept = ctypes.c_int64()
    _check(lib().pairdiag_truncate(h, dimension_limit, bins, ctypes.byref(kept)))
    return kept.value


def pairdiag_kept_map_dev(h, out) -> None:
    """Kept index of every full-space state (-1 dropped) into an int32 device tensor."""
    import torch
    if out.numel() < pairdiag_full_dim(h):
        raise ValueError("out must hold C(omega, n_pairs) elements")
    _check(lib().pairdiag_kept_map_dev(h, _dev_ptr(out, torch.int32)))


def pairdiag_basis(h) -> np.ndarray:
    out = np.empty(pairdiag_full_dim(h), dtype=np.uint64)
    _check(lib().pairdiag_basis(h, _np_ptr(out)))
    return out


def pairdiag_basis_dev(h, first: int, count: int, out) -> None:
    import torch
    if out.numel() < count:
        raise ValueError(f"out has {out.numel()} elements, fewer than count = {count}")
    _check(lib().pairdiag_basis_dev(h, first, count, _dev_ptr(out, torch.int64)))


def pairdiag_rank_dev(h, states, ranks) -> None:
    import torch
    if ranks.numel() < states.numel():
        raise ValueError(f"ranks has {ranks.numel()} elements, fewer than the {states.numel()} states")
    _check(lib().pairdiag_rank_dev(h, _dev_ptr(states, torch.int64), states.numel(), _dev_ptr(ranks, torch.int64)))


def pairdiag_hx_dev(h, precision: int, x, y) -> None:
    """y = H x on device tensors: PD_PREC_FP64 (double x, y), PD_PREC_MIXED
    (float x, y) or PD_HX_FLOATFLOAT (float x, double y)."""
    import torch
    if precision == PD_HX_FLOATFLOAT:
        dx, dy = torch.float32, torch.float64
    else:
        dx = dy = torch.float64 if precision == PD_PREC_FP64 else torch.float32
    dim = pairdiag_dim(h)
    if x.numel() < dim or y.numel() < dim:
        raise ValueError(f"x and y need dim = {dim} elements")
    _check(lib().pairdiag_hx_dev(h, precision, _dev_ptr(x, dx), _dev_ptr(y, dy)))


def pairdiag_hx(h, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.size != pairdiag_dim(h):
        raise ValueError("x must hold dim elements")
    y = np.empty_like(x)
    _check(lib().pairdiag_hx(h, _np_ptr(x), _np_ptr(y)))
    return y


def pairdiag_monopole(h):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    pos = ctypes.c_int64()
    _check(lib().pairdiag_monopole(h, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(pos)))
    return lo.value, hi.value, pos.value


def pairdiag_set_start(h, v) -> None:
    v = np.ascontiguousarray(v, dtype=np.float64)
    if v.size != pairdiag_dim(h):
        raise ValueError("v must hold dim elements")
    _check(lib().pairdiag_set_start(h, _np_ptr(v)))


def pairdiag_ground_state(h, tol: float, want_vector: bool = True, out: np.ndarray | None = None) -> dict:
    """out (optional): a float64 host array of dim elements that receives the
    eigenvector (pinned memory makes the copy faster); by default one is made."""
    e0 = ctypes.c_double()
    info = pairdiag_info()
    if want_vector and out is not None:
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != pairdiag_dim(h):
            raise ValueError("out must be a contiguous float64 array of dim elements")
        vec = out
    else:
        vec = np.empty(pairdiag_dim(h), dtype=np.float64) if want_vector else None
    st = _check(lib().pairdiag_ground_state(h, tol, ctypes.byref(e0), _np_ptr(vec) if want_vector else None,
                                            ctypes.byref(info)), allow=(PD_OK, PD_ENOCONV))
    return dict(e0=e0.value, vec=vec, status=st, **info.as_dict())


def pairdiag_ground_state_dev(h, tol: float, vec=None) -> dict:
    import torch
    e0 = ctypes.c_double()
    info = pairdiag_info()
    if vec is not None and vec.numel() < pairdiag_dim(h):
        raise ValueError("vec must hold dim elements")
    st = _check(lib().pairdiag_ground_state_dev(h, tol, ctypes.byref(e0),
                                                _dev_ptr(vec, torch.float64) if vec is not None else None,
                                                ctypes.byref(info)), allow=(PD_OK, PD_ENOCONV))
    return dict(e0=e0.value, status=st, **info.as_dict())


def pairdiag_lowest_states_dev(h, k: int, tol: float, vecs=None) -> dict:
    """The k lowest eigenpairs by locking.  vecs: optional float64 device tensor of
    k * dim elements (state j at row j).  Returns energies [k], status and the
    per-state info records."""
    import torch
    if vecs is not None and vecs.numel() < k * pairdiag_dim(h):
        raise ValueError("vecs must hold k * dim elements")
    energies = np.empty(max(k, 1))
    infos = (pairdiag_info * max(k, 1))()
    st = _check(lib().pairdiag_lowest_states_dev(h, k, tol, _np_ptr(energies),
                                                 _dev_ptr(vecs, torch.float64) if vecs is not None else None,
                                                 ctypes.cast(infos, ctypes.POINTER(pairdiag_info))),
                allow=(PD_OK, PD_ENOCONV))
    return dict(energies=energies[:k], status=st, info=[i.as_dict() for i in infos][:k])


def pairdiag_occupations_dev(h, v, omega: int) -> np.ndarray:
    """Occupation numbers 2<v|S+_i S-_i|v> of the first ``omega`` orbits."""
    import torch
    if v.numel() < pairdiag_dim(h):
        raise ValueError("v must hold dim elements")
    out = np.empty(64, dtype=np.float64)
    _check(lib().pairdiag_occupations_dev(h, _dev_ptr(v, torch.float64), _np_ptr(out)))
    return out[:omega].copy()


def _multidot_args(Q, ld: int, m: int, p, n: int, out=None) -> int:
    """Checks the sizes and types of a multi-dot before any pointer reaches the
    library, which cannot see them: Q holds m vectors of n elements at stride
    ld, p holds n elements, out (when given) m float64 values on Q's device.
    Returns the library's dtype code (0 double, 1 float)."""
    import torch
    if Q.dtype not in (torch.float64, torch.float32):
        raise TypeError(f"Q must be float64 or float32, got {Q.dtype}")
    if p.dtype != Q.dtype:
        raise TypeError(f"p must have Q's dtype {Q.dtype}, got {p.dtype}")
    if m < 1 or n < 0 or ld < n:
        raise ValueError(f"need m >= 1 and 0 <= n <= ld (m={m}, n={n}, ld={ld})")
    if Q.numel() < (m - 1) * ld + n:
        raise ValueError(f"Q has {Q.numel()} elements, fewer than (m-1)*ld+n = {(m - 1) * ld + n}")
    if p.numel() < n:
        raise ValueError(f"p has {p.numel()} elements, fewer than n = {n}")
    if p.device != Q.device:
        raise ValueError("p must be on Q's device")
    if out is not None:
        if out.dtype != torch.float64:
            raise TypeError(f"out must be float64, got {out.dtype}")
        if out.numel() < m:
            raise ValueError(f"out has {out.numel()} elements, fewer than m = {m}")
        if out.device != Q.device:
            raise ValueError("out must be on Q's device")
    return 0 if Q.dtype == torch.float64 else 1


def pairdiag_fma_peak(precision: int, reps: int = 5, stream=None) -> float:
    """Measured FMA throughput (TFLOP/s, 2 flops per FMA) of the current device in
    FP64 (PD_PREC_FP64) or FP32 (PD_PREC_MIXED)."""
    out = ctypes.c_double()
    sp = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().pairdiag_fma_peak(precision, reps, ctypes.c_void_p(sp), ctypes.byref(out)))
    return out.value


def pairdiag_multidot(h, Q, ld: int, m: int, p, n: int) -> np.ndarray:
    dtype = _multidot_args(Q, ld, m, p, n)
    out = np.empty(m, dtype=np.float64)
    _check(lib().pairdiag_multidot(h, dtype, _dev_ptr(Q), ld, m, _dev_ptr(p, Q.dtype), n, _np_ptr(out)))
    return out


def pairdiag_multidot_noalloc(Q, ld: int, m: int, p, n: int, out, stream=None) -> None:
    """Allocation-free multi-dot (no handle): out[j] = Q[j] . p in FP64, written to
    the device tensor ``out`` (float64, m elements) on ``stream``."""
    import torch
    dtype = _multidot_args(Q, ld, m, p, n, out)
    sp = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().pairdiag_multidot_noalloc(dtype, _dev_ptr(Q), ld, m, _dev_ptr(p, Q.dtype), n,
                                           _dev_ptr(out, torch.float64), ctypes.c_void_p(sp)))


def pairdiag_batch_ground_state(problems, tol: float, opt: pairdiag_options | None = None, stream=None,
                                mlp=None) -> dict:
    """problems: sequence of (omega, n_pairs, e, G).  Returns per-problem arrays
    e0, status, iterations, converged, stalled, rel_residual, latency_ms and the
    call's status."""
    count = len(problems)
    if count < 1:
        raise ValueError("need at least one problem")
    om = np.array([p[0] for p in problems], dtype=np.int32)
    nn = np.array([p[1] for p in problems], dtype=np.int32)
    es = [np.asarray(p[2], dtype=np.float64) for p in problems]
    Gs = [np.asarray(p[3], dtype=np.float64) for p in problems]
    # the library finds problem i's e and G at the running sums of omega and
    # omega^2, so every shape must match its omega
    for i, (o, e, G) in enumerate(zip(om, es, Gs)):
        if e.shape != (o,) or G.shape != (o, o):
            raise ValueError(f"problem {i}: e must be [omega] and G [omega, omega] (omega = {o})")
    e_all = np.ascontiguousarray(np.concatenate([e.ravel() for e in es]))
    G_all = np.ascontiguousarray(np.concatenate([G.ravel() for G in Gs]))
    e0 = np.empty(count)
    status = np.empty(count, dtype=np.int32)
    res = (pairdiag_batch_result * count)()
    sp = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    st = _check(lib().pairdiag_batch_ground_state(count, _np_ptr(om), _np_ptr(nn), _np_ptr(e_all), _np_ptr(G_all),
                                                  tol, ctypes.byref(opt) if opt is not None else None, mlp,
                                                  _np_ptr(e0), _np_ptr(status), ctypes.cast(res, ctypes.c_void_p),
                                                  ctypes.c_void_p(sp)), allow=(PD_OK, PD_ENOCONV))
    out = dict(e0=e0, status=status, call_status=st)
    for f, _ in pairdiag_batch_result._fields_:
        out[f] = np.array([getattr(r, f) for r in res])
    return out


def pairdiag_odd_ground_state(omega: int, n_pairs: int, e, G, tol: float, block: int = -1,
                              opt: pairdiag_options | None = None, mlp=None, want_vector: bool = True) -> dict:
    """Odd-mass ground state with one blocked orbit (block -1: every orbit, the
    lowest returned).  Returns e0, block, energies [omega] (NaN where not
    solved), occ [omega], vec (pair vector on the other orbits, or None), the
    winning subspace's info fields and the call's status."""
    e = np.ascontiguousarray(e, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    if e.shape != (omega,) or G.shape != (omega, omega):
        raise ValueError("e must be [omega] and G [omega, omega]")
    e0 = ctypes.c_double()
    b_out = ctypes.c_int()
    energies = np.empty(omega)
    occ = np.empty(omega)
    vec = None
    if want_vector and 0 <= n_pairs < omega:
        from math import comb
        vec = np.empty(comb(omega - 1, n_pairs))
    info = pairdiag_info()
    st = _check(lib().pairdiag_odd_ground_state(omega, n_pairs, _np_ptr(e), _np_ptr(G), block, tol,
                                                ctypes.byref(opt) if opt is not None else None, mlp,
                                                ctypes.byref(e0), ctypes.byref(b_out), _np_ptr(energies),
                                                _np_ptr(occ), _np_ptr(vec) if vec is not None else None,
                                                ctypes.byref(info)), allow=(PD_OK, PD_ENOCONV))
    return dict(e0=e0.value, block=b_out.value, energies=energies, occ=occ, vec=vec, status=st,
                **info.as_dict())


def pairdiag_tridiag_lowest(h, alpha, beta):
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    if alpha.ndim != 1 or beta.ndim != 1:
        raise ValueError("alpha and beta must be 1-D")
    m = len(alpha)
    if m < 1 or beta.size < m - 1:
        raise ValueError(f"need m >= 1 diagonal entries and m - 1 off-diagonal ones (m = {m}, beta {beta.size})")
    theta = np.empty(2)
    s = np.empty(m)
    _check(lib().pairdiag_tridiag_lowest(h, m, _np_ptr(alpha), _np_ptr(beta) if m > 1 else None,
                                         _np_ptr(theta), _np_ptr(s)))
    return theta, s


def pairdiag_kernel_launches() -> int:
    return int(lib().pairdiag_kernel_launches())


def pairdiag_release_cache() -> int:
    """Return the library's cached device blocks to the driver; their bytes."""
    n = ctypes.c_size_t()
    _check(lib().pairdiag_release_cache(ctypes.byref(n)))
    return n.value


def pairdiag_set_profiling(h, on: bool) -> None:
    _check(lib().pairdiag_set_profiling(h, 1 if on else 0))


def pairdiag_set_step_fusion(h, on: bool) -> None:
    """One cooperative launch per Lanczos step (True, default) or three launches."""
    _check(lib().pairdiag_set_step_fusion(h, 1 if on else 0))


PD_PROF_STEP = 2     # record kinds PD_PROF_STEP + PD_PREC_*: the Lanczos steps' vector work


def pairdiag_get_profile(h, precision: int = PD_PREC_MIXED):
    """(number of timed regions of this kind, their summed duration in ms);
    clears the records returned.  Kinds: PD_PREC_FP64 / PD_PREC_MIXED H*x
    launches (negative: both), PD_PROF_STEP + PD_PREC_* the steps' vector work."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(lib().pairdiag_get_profile(h, precision, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


# ------------------------------------------------------- learned warm start ---
def pairdiag_mlp_create(seed: int = 0):
    m = _H()
    _check(lib().pairdiag_mlp_create(seed, ctypes.byref(m)))
    return m


def pairdiag_mlp_destroy(m) -> None:
    lib().pairdiag_mlp_destroy(m)


def pairdiag_mlp_num_params() -> int:
    return int(lib().pairdiag_mlp_num_params())


def pairdiag_mlp_get_params(m) -> np.ndarray:
    out = np.empty(pairdiag_mlp_num_params(), dtype=np.float32)
    _check(lib().pairdiag_mlp_get_params(m, _np_ptr(out)))
    return out


def pairdiag_mlp_set_params(m, theta) -> None:
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    if theta.size != pairdiag_mlp_num_params():
        raise ValueError(f"theta must hold {pairdiag_mlp_num_params()} parameters, not {theta.size}")
    _check(lib().pairdiag_mlp_set_params(m, _np_ptr(theta)))


def pairdiag_mlp_features(omega: int, n_pairs: int, e, G) -> np.ndarray:
    e = np.ascontiguousarray(e, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    X = np.empty((omega, 16), dtype=np.float32)
    _check(lib().pairdiag_mlp_features(omega, n_pairs, _np_ptr(e), _np_ptr(G), _np_ptr(X)))
    return X


def _feature_rows(X, target=None):
    """X as a contiguous float32 [rows, 16] array (and target as float32 [rows]):
    the library reads rows * 16 and rows floats from them."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2 or X.shape[1] != 16:
        raise ValueError(f"X must be [rows, 16] feature rows, not {X.shape}")
    if target is None:
        return X
    t = np.ascontiguousarray(target, dtype=np.float32)
    if t.shape != (len(X),):
        raise ValueError(f"target must be [{len(X)}], not {t.shape}")
    return X, t


def pairdiag_mlp_forward(m, X) -> np.ndarray:
    X = _feature_rows(X)
    out = np.empty(len(X), dtype=np.float32)
    _check(lib().pairdiag_mlp_forward(m, len(X), _np_ptr(X), _np_ptr(out)))
    return out


def pairdiag_mlp_loss_grad(m, X, target):
    X, t = _feature_rows(X, target)
    loss = ctypes.c_double()
    grad = np.empty(pairdiag_mlp_num_params(), dtype=np.float32)
    _check(lib().pairdiag_mlp_loss_grad(m, len(X), _np_ptr(X), _np_ptr(t), ctypes.byref(loss), _np_ptr(grad)))
    return loss.value, grad


def pairdiag_mlp_buffer(m, which: int, rows: int) -> np.ndarray:
    """An intermediate of the last pass (PD_MLP_*) as float32: [rows, 128], or
    [rows] for PD_MLP_OUT and PD_MLP_DOUT."""
    n = rows if which in (PD_MLP_OUT, PD_MLP_DOUT) else rows * 128
    out = np.empty(n, dtype=np.float32)
    _check(lib().pairdiag_mlp_buffer(m, which, rows, _np_ptr(out)))
    return out if which in (PD_MLP_OUT, PD_MLP_DOUT) else out.reshape(rows, 128)


def pairdiag_mlp_train(m, X, target, steps: int, lr: float = 1e-3) -> np.ndarray:
    X, t = _feature_rows(X, target)
    if steps < 0:
        raise ValueError("steps must be >= 0")
    hist = np.empty(steps, dtype=np.float64)
    _check(lib().pairdiag_mlp_train(m, len(X), _np_ptr(X), _np_ptr(t), steps, lr, _np_ptr(hist)))
    return hist


def pairdiag_set_mlp(h, m) -> None:
    _check(lib().pairdiag_set_mlp(h, m))


def _orbit_weights(h, w):
    """w as a contiguous float64 [omega] array for the handle's omega (the
    library reads omega doubles from it)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    omega = pairdiag_omega(h)
    if omega < 1:
        raise ValueError("not a valid handle")
    if w.shape != (omega,):
        raise ValueError(f"w must be [{omega}] (one weight per orbit), not {w.shape}")
    return w


def pairdiag_set_start_weights(h, w) -> None:
    w = _orbit_weights(h, w)
    _check(lib().pairdiag_set_start_weights(h, _np_ptr(w)))


def pairdiag_product_fit(h, v, omega: int) -> np.ndarray:
    import torch
    if v.numel() < pairdiag_dim(h):
        raise ValueError("v must hold dim elements")
    w = np.empty(64, dtype=np.float64)
    _check(lib().pairdiag_product_fit(h, _dev_ptr(v, torch.float64), _np_ptr(w)))
    return w[:omega].copy()


def pairdiag_product_start_dev(h, w, v) -> None:
    import torch
    w = _orbit_weights(h, w)
    if v.numel() < pairdiag_dim(h):
        raise ValueError("v must hold dim elements")
    _check(lib().pairdiag_product_start_dev(h, _np_ptr(w), _dev_ptr(v, torch.float64)))


# ---------------------------------------------------------------- autotuner ---
def pairdiag_autotune(omega: int, n_pairs: int, e, G, precision: int = PD_PREC_MIXED, reps: int = 5):
    """Time every (low_bits, hx_variant) candidate; returns (best, all) as dicts."""
    e = np.ascontiguousarray(e, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    best = pairdiag_tune_entry()
    cap = 64                                  # 6 block splits x 5 variants fit
    arr = (pairdiag_tune_entry * cap)()
    n = ctypes.c_int(cap)
    _check(lib().pairdiag_autotune(omega, n_pairs, _np_ptr(e), _np_ptr(G), precision, reps, ctypes.byref(best),
                                   ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(n)))
    as_d = lambda t: {"low_bits": t.low_bits, "hx_variant": t.hx_variant, "ms": t.ms}
    return as_d(best), [as_d(arr[i]) for i in range(n.value)]


def pairdiag_tune_set(omega: int, n_pairs: int, precision: int, low_bits: int, hx_variant: int = 1) -> None:
    _check(lib().pairdiag_tune_set(omega, n_pairs, precision, low_bits, hx_variant))


def pairdiag_tune_get(omega: int, n_pairs: int, precision: int):
    lb, hv = ctypes.c_int(), ctypes.c_int()
    _check(lib().pairdiag_tune_get(omega, n_pairs, precision, ctypes.byref(lb), ctypes.byref(hv)))
    return lb.value, hv.value


# ------------------------------------------------------------ convenience ---
class Solver:
    """RAII wrapper: ``with Solver(omega, n, e, G, precision=...) as s: s.ground_state(1e-10)``."""

    def __init__(self, omega: int, n_pairs: int, e, G, **options):
        self.omega, self.n_pairs = omega, n_pairs
        self.h = pairdiag_create(omega, n_pairs, e, G, pairdiag_default_options(**options))

    @property
    def dim(self) -> int:
        return pairdiag_dim(self.h)

    @property
    def nnz(self) -> int:
        return pairdiag_nnz(self.h)

    def ground_state(self, tol: float, want_vector: bool = True, out: np.ndarray | None = None) -> dict:
        return pairdiag_ground_state(self.h, tol, want_vector, out)

    def close(self):
        if self.h is not None:
            pairdiag_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

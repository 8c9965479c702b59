"""GB300-native (sm_103a) ground-state solver for the general pairing
Hamiltonian in the seniority-zero basis (the method of Liu & Qi, "PairDiag").

The computation lives in libpairdiag.so (CUDA, C ABI in include/pairdiag.h);
``pairdiag`` is its ctypes binding.
"""
from .pairdiag import *  # noqa: F401,F403
from .pairdiag import Solver, lib, library_path, exported_symbols  # noqa: F401

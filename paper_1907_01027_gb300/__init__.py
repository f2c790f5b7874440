"""GB300-native low-memory S_N-DG transport sweeps (Sun & Hauck, arXiv 1907.01027).

The compute path is ``liblmdg.so`` (hand-written CUDA for sm_103a, C ABI in ``include/lmdg.h``); this package
is a thin ctypes binding over it.  There is no CPU fallback: importing :mod:`.lmdg` raises if the library is
not built.
"""
from .lmdg import (Context, LmdgError, build, STD, LM, RLM, P0, FP64, FP32, FP32_BF16STORE, SWEEP_SOURCE,
                   SWEEP_FP32, SWEEP_STORE, SWEEP_F32X2, SOLVE_EXACT_REF, HOST_PTRS, RESID_FP64, RESID_F32X2, VARIANTS)

__all__ = ["Context", "LmdgError", "build", "STD", "LM", "RLM", "P0", "FP64", "FP32", "FP32_BF16STORE",
           "SWEEP_SOURCE", "SWEEP_FP32", "SWEEP_STORE", "SWEEP_F32X2", "SOLVE_EXACT_REF", "HOST_PTRS", "RESID_FP64", "RESID_F32X2",
           "VARIANTS"]

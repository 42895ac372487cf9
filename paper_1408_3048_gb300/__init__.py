"""GB300-native GLS map-making: PCG for (P^T N^-1 P) m = P^T N^-1 d with block-Jacobi
and two-level (deflation) preconditioning, after Szydlarski, Grigori & Stompor,
arXiv 1408.3048.

The compute path is the C-ABI library ``libmm.so`` (hand-written sm_103a CUDA kernels,
declared in ``include/mm.h``); ``paper_1408_3048_gb300.mm`` is its thin ctypes binding.
Importing this package does not load the library; the first call into ``mm`` does, and
raises if it is missing (there is no CPU fallback).
"""
__all__ = ["mm", "synth"]

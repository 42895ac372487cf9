"""Block-diagonal banded Toeplitz N^-1 (Eq. 4; band of Sec. 4.1.4) -- oracle.

N^-1 = diag(T_0, ..., T_K): block i acts on the samples of stationary interval i only
(size t_i x t_i, no wrap-around, no coupling between intervals).  T_i is symmetric
Toeplitz with first row (t^(i)_0, ..., t^(i)_lambda, 0, ...), so for t in interval i

    z_t = sum_{|k| <= lambda, t+k in interval i} t^(i)_{|k|} y_{t+k}.

Three independent routes: direct convolution (the definition), a dense matrix (tiny
blocks) and FFT convolution (large blocks).  Test infrastructure only.
"""
import numpy as np
import scipy.linalg
import scipy.signal


def _full_kernel(t):
    t = np.asarray(t, dtype=np.float64)
    return np.concatenate([t[:0:-1], t])  # t_lam .. t_1, t_0, t_1 .. t_lam


def apply_block_direct(y, t):
    """z = T y for one block of Eq. 4 by direct convolution (np.convolve is the plain sum;
    band |k| <= lambda of Sec. 4.1.4, truncated at the block edges: readings R3, R5)."""
    lam = len(t) - 1
    full = np.convolve(np.asarray(y, dtype=np.float64), _full_kernel(t), mode="full")
    return full[lam : lam + len(y)]


def apply_block_fft(y, t):
    """The same product (one block of Eq. 4) through scipy.signal.fftconvolve (library FFT
    as a step)."""
    lam = len(t) - 1
    full = scipy.signal.fftconvolve(np.asarray(y, dtype=np.float64), _full_kernel(t), mode="full")
    return full[lam : lam + len(y)]


def dense_block(t, n):
    """T as a dense n x n symmetric Toeplitz matrix (one block of Eq. 4, band truncated at
    the block edge)."""
    c = np.zeros(n, dtype=np.float64)
    m = min(n, len(t))
    c[:m] = t[:m]
    return scipy.linalg.toeplitz(c)


def apply_ninv(y, offsets, interval_psd, rows, route="direct"):
    """z = N^-1 y over all intervals (Eq. 4: block-diagonal, one block per stationary
    interval).  offsets[K+1], interval_psd[K], rows[psd] = t_k."""
    y = np.asarray(y, dtype=np.float64)
    z = np.zeros_like(y)
    fn = apply_block_direct if route == "direct" else apply_block_fft
    for i in range(len(offsets) - 1):
        a, b = int(offsets[i]), int(offsets[i + 1])
        z[a:b] = fn(y[a:b], rows[int(interval_psd[i])])
    return z


def dense_ninv(offsets, interval_psd, rows):
    """N^-1 of Eq. 4 as a dense block-diagonal matrix (tiny problems only)."""
    blocks = [
        dense_block(rows[int(interval_psd[i])], int(offsets[i + 1] - offsets[i]))
        for i in range(len(offsets) - 1)
    ]
    return scipy.linalg.block_diag(*blocks)


def diagonal(nt, offsets, interval_psd, rows):
    """diag(N^-1): t^(i(t))_0 for every sample (used by M_BD, Eq. 10)."""
    d = np.empty(nt, dtype=np.float64)
    for i in range(len(offsets) - 1):
        d[int(offsets[i]) : int(offsets[i + 1])] = rows[int(interval_psd[i])][0]
    return d

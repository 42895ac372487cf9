"""Noise model -> banded Toeplitz rows of N^-1 (oracle; test infrastructure only).

Paper facts used:
  * Eq. 19 (Sec. 4.1.4): the noise PSD of a stationary piece is
    P(f) = sigma^2 t_samp (1 + (f_knee / f)^2).  The exponent 2 is generalised to alpha.
  * Sec. 2.1: each diagonal block of N^-1 is a symmetric Toeplitz matrix; App. D: one
    row of that block is the Fourier transform of the inverse PSD.
  * Sec. 4.1.4: the blocks are band-diagonal, correlations beyond the half bandwidth
    lambda_T are zero.
  * App. D, Eq. 28: band-diagonality is imposed by apodising the row with a Gaussian
    window that vanishes beyond lambda_T.

Readings where the paper is silent or garbled (the same readings are listed in the
design notes and implemented independently by the CUDA library):
  R1  Discrete spectrum on a grid of L = 2^ceil(log2(max interval length)) points,
      f_j = j f_s / L, S_j = sigma^2 (1 + (f_knee/f_j)^alpha) for j >= 1 (the t_samp of
      Eq. 19 is divided out, so white noise gives t_0 = 1/sigma^2).  1/S_0 is the
      f -> 0 limit: 0 when f_knee > 0, 1/sigma^2 when f_knee = 0.
      r_k = (1/L) sum_{j=0}^{L-1} S_{min(j, L-j)}^-1 cos(2 pi j k / L).
  R2  Eq. 28 is printed without its minus sign; window w_k = exp(-2 (k/lambda)^2) for
      |k| <= lambda, 0 beyond (GAUSS).  RECT (w_k = 1) is provided for dense tests.
  R3  Half bandwidth lambda: the nonzero lags are |k| <= lambda (2 lambda + 1 diagonals).
  R4  Positive definiteness: the symbol t_0 + 2 sum_k t_k cos(w k) is evaluated on
      M = 2^ceil(log2(max(8 lambda, 8))) equispaced frequencies; the row is rejected
      when its minimum is <= 0.
"""
import numpy as np

WINDOW_GAUSS = 0
WINDOW_RECT = 1


def grid_length(interval_lengths):
    """R1: L = 2^ceil(log2(max_i t_i)) (at least 2)."""
    m = int(max(int(v) for v in interval_lengths))
    L = 1
    while L < m:
        L *= 2
    return max(L, 2)


def inverse_psd_grid(sigma, fknee, alpha, L, fsamp):
    """R1: 1/S_j for j = 0..L/2 (Eq. 19 with exponent alpha, t_samp divided out)."""
    j = np.arange(L // 2 + 1, dtype=np.float64)
    f = j * fsamp / L
    inv = np.empty(L // 2 + 1, dtype=np.float64)
    with np.errstate(divide="ignore"):
        S = sigma * sigma * (1.0 + (fknee / f[1:]) ** alpha)
    inv[1:] = 1.0 / S
    inv[0] = 0.0 if fknee > 0.0 else 1.0 / (sigma * sigma)
    return inv


def row_direct(inv_psd, L, lam):
    """R1 by the plain cosine sum over all L grid frequencies: r_k, k = 0..lam.

    O(L * lam); used for small grids and to pin the FFT route."""
    sym = inv_psd[np.minimum(np.arange(L), L - np.arange(L))]
    r = np.empty(lam + 1, dtype=np.float64)
    for k in range(lam + 1):
        # cos(2 pi j k / L) with the argument reduced exactly in integers first
        ang = 2.0 * np.pi * ((np.arange(L, dtype=np.int64) * k) % L) / L
        r[k] = np.dot(sym, np.cos(ang)) / L
    return r


def row_fft(inv_psd, L, lam):
    """R1 by the inverse real FFT of the Hermitian-symmetric grid (numpy.fft as a step)."""
    r = np.fft.irfft(inv_psd, n=L)
    return r[: lam + 1].copy()


def window(lam, kind=WINDOW_GAUSS):
    """R2: apodisation window w_k, k = 0..lam (Eq. 28 with the sign restored)."""
    k = np.arange(lam + 1, dtype=np.float64)
    if kind == WINDOW_RECT:
        return np.ones(lam + 1)
    if lam == 0:
        return np.ones(1)
    return np.exp(-2.0 * (k / lam) ** 2)


def toeplitz_row(sigma, fknee, alpha, L, fsamp, lam, kind=WINDOW_GAUSS, route="fft"):
    """t_k = w_k r_k, k = 0..lam: the first row of one banded Toeplitz block of N^-1
    (App. D and Eq. 28 by readings R1-R3)."""
    inv = inverse_psd_grid(sigma, fknee, alpha, L, fsamp)
    r = row_fft(inv, L, lam) if route == "fft" else row_direct(inv, L, lam)
    return window(lam, kind) * r


def symbol_grid_size(lam):
    """R4: number of frequencies M on which the symbol is checked."""
    m = max(8 * lam, 8)
    M = 1
    while M < m:
        M *= 2
    return M


def symbol(t, M):
    """sigma(w_m) = t_0 + 2 sum_{k>=1} t_k cos(w_m k), w_m = 2 pi m / M, m = 0..M-1: the
    symbol of the banded block, whose minimum decides positive definiteness (reading R4)."""
    lam = len(t) - 1
    m = np.arange(M, dtype=np.int64)
    s = np.full(M, t[0], dtype=np.float64)
    for k in range(1, lam + 1):
        s += 2.0 * t[k] * np.cos(2.0 * np.pi * ((m * k) % M) / M)
    return s


def symbol_fft(t, M):
    """The same M symbol values by one real FFT of the even row laid out circularly
    (reading R4)."""
    lam = len(t) - 1
    h = np.zeros(M, dtype=np.float64)
    h[0] = t[0]
    h[1 : lam + 1] = t[1:]
    if lam > 0:
        h[M - lam :] = t[1:][::-1]
    return np.fft.fft(h).real


def is_positive_definite(t):
    """R4: True when min symbol > 0 (then every finite section of the band is SPD)."""
    lam = len(t) - 1
    M = symbol_grid_size(lam)
    s = symbol(t, M) if lam <= 256 else symbol_fft(t, M)
    return bool(s.min() > 0.0)

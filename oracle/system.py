"""The GLS system A m = b of Eq. 5-8 (oracle; test infrastructure only).

A = P^T N^-1 P (Eq. 5) applied matrix-free from right to left (Eq. 8):
de-pointing P x, noise weighting N^-1 y, pointing P^T z.  b = P^T N^-1 d (Eq. 7).
"""
import numpy as np

from . import noise, pointing, toeplitz


class NotSPDError(ValueError):
    """A banded Toeplitz row whose symbol is not positive (reading R4)."""


class Problem:
    """Plan + operators of one map-making problem.

    pix[nt]            sky pixel of every sample (0 <= pix < npix_sky)
    weights[nt, 2]     (cos 2 phi_t, sin 2 phi_t) for ncomp = 3, else None
    offsets[K+1]       interval boundaries, offsets[0] = 0, offsets[K] = nt, increasing
    interval_psd[K]    PSD id of every interval
    psds[npsd]         (sigma, fknee, alpha) per PSD id (Eq. 19)
    lam                half bandwidth (0 <= lam < shortest interval)
    """

    def __init__(self, pix, npix_sky, weights, offsets, interval_psd, psds, fsamp, lam,
                 ncomp, window=noise.WINDOW_GAUSS, rcond_min=1e-6, row_route="fft",
                 check_spd=True):
        self.pix = np.asarray(pix, dtype=np.int64)
        self.nt = self.pix.size
        self.npix_sky = int(npix_sky)
        self.ncomp = int(ncomp)
        if self.ncomp not in (1, 3):
            raise ValueError("ncomp must be 1 or 3")
        self.weights = None if weights is None else np.asarray(weights, dtype=np.float64).reshape(-1, 2)
        if self.ncomp == 3 and self.weights is None:
            raise ValueError("polarisation needs weights")
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.interval_psd = np.asarray(interval_psd, dtype=np.int64)
        K = self.offsets.size - 1
        if K < 1 or self.offsets[0] != 0 or self.offsets[-1] != self.nt or np.any(np.diff(self.offsets) <= 0):
            raise ValueError("bad interval offsets")
        if self.interval_psd.size != K:
            raise ValueError("interval_psd must have K entries")
        self.psds = [tuple(float(v) for v in p) for p in psds]
        if self.interval_psd.min() < 0 or self.interval_psd.max() >= len(self.psds):
            raise ValueError("psd id out of range")
        lengths = np.diff(self.offsets)
        self.lam = int(lam)
        if self.lam < 0 or self.lam >= lengths.min():
            raise ValueError("lambda must satisfy 0 <= lambda < shortest interval")
        self.fsamp = float(fsamp)
        self.L = noise.grid_length(lengths)
        self.rows = [
            noise.toeplitz_row(s, fk, a, self.L, self.fsamp, self.lam, window, route=row_route)
            for (s, fk, a) in self.psds
        ]
        if check_spd:
            for r in self.rows:
                if not noise.is_positive_definite(r):
                    raise NotSPDError("Toeplitz row is not positive definite")
        self.obs2sky, self.hits, self.pix_c = pointing.observed_pixels(
            self.pix, self.npix_sky, self.ncomp, self.weights, rcond_min)
        self.npix_obs = self.obs2sky.size
        self.n = self.npix_obs * self.ncomp

    # ---- operators (Eq. 8) -------------------------------------------------------
    def P(self, x):
        """y = P x (Eq. 2)."""
        return pointing.depoint(x, self.pix_c, self.ncomp, self.weights)

    def PT(self, y):
        """w = P^T y (Sec. 2)."""
        return pointing.point(y, self.pix_c, self.npix_obs, self.ncomp, self.weights)

    def Ninv(self, y, route="direct"):
        """z = N^-1 y (Eq. 4)."""
        return toeplitz.apply_ninv(y, self.offsets, self.interval_psd, self.rows, route)

    def A(self, x, route="direct"):
        """A x = P^T [N^-1 [P x]] (Eq. 8)."""
        return self.PT(self.Ninv(self.P(x), route))

    def rhs(self, d, route="direct"):
        """b = P^T N^-1 d (Eq. 7)."""
        return self.PT(self.Ninv(d, route))

    def ninv_diag(self):
        """diag(N^-1), the weights of M_BD (Eq. 10)."""
        return toeplitz.diagonal(self.nt, self.offsets, self.interval_psd, self.rows)

    # ---- dense forms (tiny problems only) ----------------------------------------
    def dense_P(self):
        """P (Eq. 1-2) as a dense matrix."""
        return pointing.dense_pointing(self.pix_c, self.npix_obs, self.ncomp, self.weights)

    def dense_Ninv(self):
        """N^-1 (Eq. 4) as a dense matrix."""
        return toeplitz.dense_ninv(self.offsets, self.interval_psd, self.rows)

    def dense_A(self):
        """A = P^T N^-1 P (Eq. 5) as a dense matrix."""
        P = self.dense_P()
        return P.T @ self.dense_Ninv() @ P

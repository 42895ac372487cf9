"""Pointing matrix P of Eq. 1-2 (oracle; test infrastructure only).

One row of P per time sample t: the single entry 1 at the observed pixel p_t for a
total-intensity (T) experiment, or the three entries (1, cos 2 phi_t, sin 2 phi_t) at the
(I, Q, U) columns of p_t for a polarisation-sensitive one (Eq. 2).  Sec. 2 restricts the
map to the pixels that are actually observed so that P has full column rank.

Naming follows Sec. 2: P x is the de-pointing (gather, time domain output); P^T y is the
pointing (scatter-add, pixel domain output).  Maps are pixel-major with the n_c Stokes
components of one pixel adjacent (the row order of Eq. 17).

Reading R6 (which pixels are "observed"):
  * T (n_c = 1): hits >= 1.
  * I/Q/U (n_c = 3): hits >= 3 and rcond(B_p) >= rcond_min for the unit-weight block
    B_p = sum_{t in p} w_t w_t^T, w_t = (1, cos 2 phi_t, sin 2 phi_t), with
    rcond = lambda_min(B_p) / lambda_max(B_p).  (A 1-norm estimate through the
    adjugate inverse is not used: for a block that is singular in exact arithmetic,
    e.g. a pixel seen at one polariser angle only, its cofactors and determinant are
    both rounding noise and their ratio is meaningless.)
  * Observed pixels keep ascending sky order.  Samples on unobserved pixels get no
    row entry (their time-domain values still enter N^-1).
"""
import numpy as np


def unit_weight_blocks(pix, weights, npix_sky):
    """B_p = sum_{t in p} w_t w_t^T, w_t = (1, cos 2phi_t, sin 2phi_t) of Eq. 2, for every
    sky pixel, shape (npix_sky, 3, 3), accumulated in float64 (the block whose
    conditioning decides which pixels are observed, reading R6)."""
    c = weights[:, 0]
    s = weights[:, 1]
    one = np.ones_like(c)
    comps = [one, c, s]
    B = np.zeros((npix_sky, 3, 3), dtype=np.float64)
    for a in range(3):
        for b in range(a, 3):
            v = np.bincount(pix, weights=comps[a] * comps[b], minlength=npix_sky)
            B[:, a, b] = v
            B[:, b, a] = v
    return B


def rcond2(B):
    """Reciprocal 2-norm condition number lambda_min / lambda_max of stacked symmetric
    3x3 blocks (eigenvalues by LAPACK's symmetric solver; 0 when lambda_max <= 0):
    the pixel acceptance test of reading R6."""
    ev = np.linalg.eigvalsh(B)
    lo, hi = ev[:, 0], ev[:, -1]
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = np.where(hi > 0.0, lo / hi, 0.0)
    return np.maximum(rc, 0.0)


def observed_pixels(pix, npix_sky, ncomp, weights=None, rcond_min=1e-6):
    """Reading R6.  Returns (obs2sky, hits, pix_c):
    obs2sky[q] = sky index of observed pixel q (ascending), hits[q] = its sample count,
    pix_c[t] = observed index of sample t or -1 when the sample is dropped."""
    pix = np.asarray(pix, dtype=np.int64)
    if pix.size and (pix.min() < 0 or pix.max() >= npix_sky):
        raise ValueError("pixel index out of range")
    hits_sky = np.bincount(pix, minlength=npix_sky)
    if ncomp == 1:
        obs = hits_sky >= 1
    else:
        B = unit_weight_blocks(pix, np.asarray(weights, dtype=np.float64), npix_sky)
        obs = (hits_sky >= 3) & (rcond2(B) >= rcond_min)
    obs2sky = np.nonzero(obs)[0].astype(np.int64)
    sky2obs = np.full(npix_sky, -1, dtype=np.int64)
    sky2obs[obs2sky] = np.arange(obs2sky.size)
    pix_c = sky2obs[pix]
    hits = hits_sky[obs2sky]
    return obs2sky, hits, pix_c


def depoint(x, pix_c, ncomp, weights=None):
    """y = P x (Eq. 2): y_t = x_I + cos 2phi_t x_Q + sin 2phi_t x_U at pixel p_t, 0 for
    dropped samples.  x has shape (npix_obs, ncomp) or (npix_obs * ncomp,)."""
    X = np.asarray(x, dtype=np.float64).reshape(-1, ncomp)
    kept = pix_c >= 0
    p = np.where(kept, pix_c, 0)
    y = X[p, 0].copy()
    if ncomp == 3:
        y += weights[:, 0] * X[p, 1] + weights[:, 1] * X[p, 2]
    y[~kept] = 0.0
    return y


def point(y, pix_c, npix_obs, ncomp, weights=None):
    """w = P^T y (the transpose of Eq. 2, Sec. 2): per observed pixel, sum over its samples
    of y_t (I) and, for polarisation, cos 2phi_t y_t (Q) and sin 2phi_t y_t (U).  Flat
    (npix_obs*ncomp,)."""
    y = np.asarray(y, dtype=np.float64)
    kept = pix_c >= 0
    p = pix_c[kept]
    yk = y[kept]
    W = np.zeros((npix_obs, ncomp), dtype=np.float64)
    W[:, 0] = np.bincount(p, weights=yk, minlength=npix_obs)
    if ncomp == 3:
        W[:, 1] = np.bincount(p, weights=weights[kept, 0] * yk, minlength=npix_obs)
        W[:, 2] = np.bincount(p, weights=weights[kept, 1] * yk, minlength=npix_obs)
    return W.reshape(-1)


def dense_pointing(pix_c, npix_obs, ncomp, weights=None):
    """P of Eq. 1-2 as a dense (nt, npix_obs*ncomp) matrix (tiny problems only)."""
    nt = pix_c.size
    P = np.zeros((nt, npix_obs * ncomp), dtype=np.float64)
    for t in range(nt):
        q = pix_c[t]
        if q < 0:
            continue
        P[t, q * ncomp] = 1.0
        if ncomp == 3:
            P[t, q * ncomp + 1] = weights[t, 0]
            P[t, q * ncomp + 2] = weights[t, 1]
    return P

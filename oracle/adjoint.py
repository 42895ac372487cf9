"""Gradients of a loss on the GLS map (oracle; test infrastructure only).

The paper gives the estimate m = (P^T N^-1 P)^-1 P^T N^-1 d (Eq. 3); it does not
differentiate it.  Differentiating Eq. 3 (A = P^T N^-1 P symmetric, Eq. 5):

  dm/dd      = A^-1 P^T N^-1              so   dL/dd = N^-1 P mu,   mu = A^-1 g
  dm/dtheta  = A^-1 P^T (dN^-1/dtheta) (d - P m)
                                          so   dL/dtheta = (P mu)^T (dN^-1/dtheta) (d - P m)

with g = dL/dm.  N^-1 depends on the PSD parameters theta = (sigma, f_knee, alpha) of
each PSD id through the Toeplitz rows (Eq. 19, App. D): the derivative rows are the
same inverse-PSD row transform applied to the analytic derivative of 1/S_j,

  d(1/S)/dsigma  = -(2/sigma) / S
  d(1/S)/dfknee  = -(1/S) alpha x / (fknee (1 + x)),   x = (fknee / f)^alpha
  d(1/S)/dalpha  = -(1/S) x ln(fknee / f) / (1 + x)

(zero at f = 0, where 1/S_0 = 0 for fknee > 0), then times the window.  For one PSD
id p, u^T T(c) v over its intervals equals sum_k c_k R_k with the interval-restricted
lagged products R_0 = sum_t u_t v_t and R_k = sum_t (u_t v_{t+k} + u_{t+k} v_t), k >= 1.
"""
import numpy as np

from . import noise, toeplitz
from .pcg import dense_solve, pcg


def inverse_psd_derivative_grids(sigma, fknee, alpha, L, fsamp):
    """d(1/S_j)/d(sigma, fknee, alpha) for j = 0..L/2 (requires fknee > 0): the analytic
    derivatives of the inverse of the Eq. 19 PSD on the grid of reading R1 (R14)."""
    if not fknee > 0.0:
        raise ValueError("the PSD gradient needs fknee > 0")
    j = np.arange(L // 2 + 1, dtype=np.float64)
    f = j * fsamp / L
    out = np.zeros((3, L // 2 + 1), dtype=np.float64)
    x = (fknee / f[1:]) ** alpha
    invS = 1.0 / (sigma * sigma * (1.0 + x))
    out[0, 1:] = -2.0 / sigma * invS
    out[1, 1:] = -invS * alpha * x / (fknee * (1.0 + x))
    out[2, 1:] = -invS * x * np.log(fknee / f[1:]) / (1.0 + x)
    return out


def row_derivatives(sigma, fknee, alpha, L, fsamp, lam, kind=noise.WINDOW_GAUSS, route="fft"):
    """dt_k/dtheta, shape (3, lam + 1), by the row transform of reading R1 and the window."""
    grids = inverse_psd_derivative_grids(sigma, fknee, alpha, L, fsamp)
    w = noise.window(lam, kind)
    fn = noise.row_fft if route == "fft" else noise.row_direct
    return np.stack([w * fn(g, L, lam) for g in grids])


def lagged_products(u, v, offsets, interval_psd, npsd, lam):
    """R[p, k], k = 0..lam: interval-restricted lagged products of u and v per PSD id
    (the blocks of Eq. 4 act within their interval only; reading R14)."""
    R = np.zeros((npsd, lam + 1), dtype=np.float64)
    for i in range(len(offsets) - 1):
        a, b = int(offsets[i]), int(offsets[i + 1])
        ui, vi = u[a:b], v[a:b]
        p = int(interval_psd[i])
        R[p, 0] += ui @ vi
        for k in range(1, min(lam, b - a - 1) + 1):
            R[p, k] += ui[:-k] @ vi[k:] + ui[k:] @ vi[:-k]
    return R


def psd_gradient(prob, u, v, kind=noise.WINDOW_GAUSS):
    """dL/dtheta[p, (sigma, fknee, alpha)] = sum_k dt_k/dtheta R[p, k] (reading R14)."""
    R = lagged_products(u, v, prob.offsets, prob.interval_psd, len(prob.psds), prob.lam)
    G = np.zeros((len(prob.psds), 3), dtype=np.float64)
    for p, (s, fk, al) in enumerate(prob.psds):
        D = row_derivatives(s, fk, al, prob.L, prob.fsamp, prob.lam, kind)
        G[p] = D @ R[p]
    return G


def gradients(prob, d, m, g, apply_M=None, tol=1e-12, maxit=10000, dense=False):
    """(dL/dd, dL/dtheta) for the loss gradient g = dL/dm at the solution m of d: the
    derivative of Eq. 3 through one solve with the symmetric A of Eq. 5 (reading R14)."""
    if dense:
        mu = dense_solve(prob.dense_A(), g)
    else:
        res = pcg(prob.A, apply_M, g, tol, maxit)
        mu = res.x
    u = prob.P(mu)
    dLdd = prob.Ninv(u)
    v = np.asarray(d, dtype=np.float64) - prob.P(m)
    return dLdd, psd_gradient(prob, u, v)


def dense_psd_gradient(prob, u, v, kind=noise.WINDOW_GAUSS):
    """The same quantity through dense derivative blocks (tiny problems): u^T dN^-1 v,
    dN^-1 block-diagonal Toeplitz as in Eq. 4 (reading R14)."""
    G = np.zeros((len(prob.psds), 3), dtype=np.float64)
    for p, (s, fk, al) in enumerate(prob.psds):
        D = row_derivatives(s, fk, al, prob.L, prob.fsamp, prob.lam, kind)
        for c in range(3):
            rows = [D[c] if q == p else np.zeros(prob.lam + 1) for q in range(len(prob.psds))]
            dN = toeplitz.dense_ninv(prob.offsets, prob.interval_psd, rows)
            G[p, c] = u @ dN @ v
    return G

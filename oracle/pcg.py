"""Solvers (oracle; test infrastructure only).

pcg          Preconditioned conjugate gradient for A x = b (Sec. 3.1).  Reading R7
             (the paper does not print its CG): Hestenes-Stiefel PCG as in Saad,
             Iterative Methods for Sparse Linear Systems, 2003, Alg. 9.1, x_0 = 0,
             beta_j = r_{j+1}^T z_{j+1} / r_j^T z_j for every preconditioner, stop when
             the recursive residual satisfies ||r_j||_2 / ||b||_2 <= tol (the relative
             residual that Sec. 5.1 plots and stops on).  The iteration count is the
             number of products A p after the initial residual.  An optional starting
             vector x0 (the A-DEF2 variant of App. B starts from Z E^-1 Z^T b) gives
             r_0 = b - A x0; the stopping test stays relative to ||b||.
dense_solve  The GLS estimate of Eq. 3 by a dense Cholesky factorisation of A
             (tiny problems).
"""
import numpy as np
import scipy.linalg


class PCGResult:
    """What one PCG run (Sec. 3.1, reading R7) leaves: the iterate, its step count, the
    relative residual history that Sec. 5.1 plots, and the step scalars and
    preconditioned residuals the Ritz construction of Sec. 3.3.2 reads."""

    def __init__(self, x, iters, converged, rel_hist, alphas, betas, zs, rzs):
        self.x = x
        self.iters = iters
        self.converged = converged
        self.rel_hist = rel_hist      # ||r_j|| / ||b|| for j = 0..iters
        self.alphas = alphas
        self.betas = betas
        self.zs = zs                  # z_j = M r_j (only when record=True)
        self.rzs = rzs                # r_j^T z_j


def pcg(apply_A, apply_M, b, tol, maxit, record=False, x0=None):
    """Preconditioned CG for A x = b (Sec. 3.1; reading R7: Hestenes-Stiefel PCG, stop on
    ||r_j|| / ||b|| <= tol, Sec. 5.1).  record=True keeps z_j and r_j^T z_j for the
    Lanczos tridiagonal of Sec. 3.3.2; x0 is the A-DEF2 start of App. B."""
    b = np.asarray(b, dtype=np.float64)
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = np.asarray(x0, dtype=np.float64).copy()
        r = b - apply_A(x)
    bn = np.linalg.norm(b)
    rel = [np.linalg.norm(r) / bn if bn > 0 else 0.0]
    alphas, betas, zs, rzs = [], [], [], []
    if bn == 0.0:
        return PCGResult(x, 0, True, rel, alphas, betas, zs, rzs)
    z = apply_M(r)
    rho = float(r @ z)
    p = z.copy()
    if record:
        zs.append(z.copy())
        rzs.append(rho)
    it = 0
    converged = False
    while it < maxit:
        q = apply_A(p)
        pq = float(p @ q)
        if not pq > 0.0:
            raise FloatingPointError("p^T A p <= 0: operator not SPD")
        alpha = rho / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        alphas.append(alpha)
        rel.append(np.linalg.norm(r) / bn)
        if rel[-1] <= tol:
            converged = True
            break
        z = apply_M(r)
        rho_new = float(r @ z)
        beta = rho_new / rho
        betas.append(beta)
        if record:
            zs.append(z.copy())
            rzs.append(rho_new)
        p = z + beta * p
        rho = rho_new
    return PCGResult(x, it, converged, rel, alphas, betas, zs, rzs)


def dense_solve(A, b):
    """m = A^-1 b by Cholesky (Eq. 3 with M = N^-1)."""
    c = scipy.linalg.cho_factor(A)
    return scipy.linalg.cho_solve(c, b)

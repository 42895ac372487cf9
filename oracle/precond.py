"""Preconditioners of Sec. 3 (oracle; test infrastructure only).

M_BD (Eq. 10)      (P^T diag(N^-1) P)^-1: one n_c x n_c block per observed pixel,
                   B_p = sum_{t in p} t^(i(t))_0 w_t w_t^T, w_t = (1, cos 2phi, sin 2phi).
R (Eq. 11)         I - A Z E^-1 Z^T with the coarse operator E = Z^T A Z.
M_2lvl (Eq. 12)    M_BD R + Z E^-1 Z^T, applied left to right as in App. C:
                   v = E^-1 (Z^T r); z = M_BD (r - (AZ) v) + Z v, with AZ and the
                   LU factors of E precomputed once (App. C, "Constructing").
Z_D (Sec. 3.3.2)   Ritz vectors of M_BD A from a first M_BD-preconditioned solve.

Reading R8 (the paper builds the Ritz pairs from GMRES/Arnoldi, Algorithm 1, and notes
that CG serves as well): CG-Lanczos.  The k smallest eigenpairs (theta, s) of the
tridiagonal T_m built from the CG step scalars,
    T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},   T_{j,j+1} = sqrt(beta_j)/alpha_j,
give Ritz vectors V_m s with Lanczos vectors v_j = (-1)^j z_j / sqrt(r_j^T z_j)
(z_j = M_BD r_j, the preconditioned CG residuals).  The selected vectors are
orthonormalised (Euclidean QR) after dropping dependent columns.
Reading R16 (the paper says nothing on dependent coarse columns; E = Z^T A Z of Eq. 12
must be invertible): the columns are taken in order and column j is dependent when its
part orthogonal to the columns kept before it (Gram-Schmidt, projected twice) has norm
below 1e-10 times the largest column norm of the matrix -- the R_jj < 1e-10 max R_jj
rule of a QR factorisation, with the scale taken from the columns themselves.  Double
projection in FP64 resolves that part to a few eps of the column norm, so an exact
duplicate (part ~1e-16) is dropped and a near-duplicate 1e-9 away is kept.
Reading R9: E is factored by LU with partial pivoting (as App. C does).

Arnoldi route (App. A, Algorithm 1; the paper's own Z_D source): the basic Arnoldi
process on B = M_BD A from w_1 = r_0 / ||r_0||, r_0 = M_BD b' (x_0 = 0), until the GMRES
residual min_y ||beta e_1 - Hbar_j y|| falls to tol * beta, m steps, or breakdown.  The
projections h_ij = (B w_j, w_i) are taken by classical Gram-Schmidt as in Algorithm 1,
with one re-orthogonalisation pass (its coefficients added to h_ij; equal in exact
arithmetic).  Ritz pairs: eigenpairs (lambda_i, v_i) of H_m, y_i = W_m v_i (Eq. A.4);
selected when |Re lambda_i| < eps_tol (Sec. 5), at most k, smallest Re first; a complex
pair contributes the real and imaginary parts of one member's vector; then the same
orthonormalisation and dropping as above.
"""
import numpy as np
import scipy.linalg

DROP_RTOL = 1e-10   # reading R16: dependence threshold relative to the largest column norm


class BlockJacobi:
    """M_BD of Eq. 10 for a oracle.system.Problem."""

    def __init__(self, prob):
        self.ncomp = prob.ncomp
        self.npix = prob.npix_obs
        dg = prob.ninv_diag()
        kept = prob.pix_c >= 0
        p = prob.pix_c[kept]
        d = dg[kept]
        nc = self.ncomp
        B = np.zeros((self.npix, nc, nc), dtype=np.float64)
        if nc == 1:
            B[:, 0, 0] = np.bincount(p, weights=d, minlength=self.npix)
        else:
            w = prob.weights[kept]
            comps = [np.ones_like(d), w[:, 0], w[:, 1]]
            for a in range(3):
                for b in range(a, 3):
                    v = np.bincount(p, weights=d * comps[a] * comps[b], minlength=self.npix)
                    B[:, a, b] = v
                    B[:, b, a] = v
        self.blocks = B
        self.inv = np.linalg.inv(B)

    def apply(self, r):
        """z = M_BD r: each pixel's block inverse applied to its components (Eq. 10)."""
        R = np.asarray(r, dtype=np.float64).reshape(self.npix, self.ncomp)
        return np.einsum("pab,pb->pa", self.inv, R).reshape(-1)

    def dense(self):
        """M_BD (Eq. 10) as a dense block-diagonal matrix."""
        return scipy.linalg.block_diag(*list(self.inv))


class TwoLevel:
    """M_2lvl of Eq. 12 for a given deflation matrix Z (n x r)."""

    def __init__(self, prob, bd, Z, route="direct"):
        self.bd = bd
        self.Z = np.asarray(Z, dtype=np.float64)
        self.AZ = np.stack([prob.A(self.Z[:, j], route) for j in range(self.Z.shape[1])], axis=1)
        self.E = self.Z.T @ self.AZ
        self.lu = scipy.linalg.lu_factor(self.E)

    def coarse(self, r):
        """v = E^-1 Z^T r (the coarse solve of Eq. 12, LU of E as in App. C)."""
        return scipy.linalg.lu_solve(self.lu, self.Z.T @ r)

    def apply(self, r):
        """z = M_2lvl r = M_BD (r - A Z v) + Z v, v = E^-1 Z^T r (Eq. 12 in the order of
        App. C)."""
        r = np.asarray(r, dtype=np.float64)
        v = self.coarse(r)
        return self.bd.apply(r - self.AZ @ v) + self.Z @ v

    def deflate(self, y):
        """R y = y - A Z E^-1 Z^T y (Eq. 11)."""
        return y - self.AZ @ self.coarse(y)

    def apply_adef2(self, r):
        """M_2lvl^(alt) r = R^T M_BD r + Z E^-1 Z^T r (App. B, Eq. B.1, the A-DEF2 form);
        R^T = I - Z E^-1 (A Z)^T because A is symmetric."""
        r = np.asarray(r, dtype=np.float64)
        y = self.bd.apply(r)
        return y - self.Z @ scipy.linalg.lu_solve(self.lu, self.AZ.T @ y) + self.Z @ self.coarse(r)

    def adef2_start(self, b):
        """The starting vector x0 = Z E^-1 Z^T b that makes A-DEF2 equivalent to an SPD
        preconditioner in exact arithmetic (App. B): Z^T r_0 = 0."""
        return self.Z @ self.coarse(b)


def lanczos_tridiagonal(alphas, betas):
    """T_m from m CG steps (alphas[0..m-1], betas[0..m-2]): the Lanczos tridiagonal of the
    first solve (Sec. 3.3.2, reading R8)."""
    m = len(alphas)
    T = np.zeros((m, m), dtype=np.float64)
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return T


def ritz_coarse_space(alphas, betas, zs, rzs, k, drop_rtol=1e-10, eps_tol=None):
    """Reading R8.  zs[j] = z_j, rzs[j] = r_j^T z_j for j = 0..m-1.
    Returns (Z with orthonormal columns, the Ritz values of the kept columns, ascending:
    the k smallest unless a dependent column was dropped).  With eps_tol the
    Ritz pairs kept are those with value below eps_tol (Sec. 5: |Re lambda_i| < eps_tol,
    the paper uses 0.2), at most k of them, smallest first."""
    m = len(alphas)
    T = lanczos_tridiagonal(alphas, betas)
    theta, S = np.linalg.eigh(T)
    kk = min(k, m)
    if eps_tol is not None:
        kk = min(kk, int(np.sum(np.abs(theta) < eps_tol)))
        if kk == 0:
            raise ValueError("no Ritz value below eps_tol")
    V = np.stack([((-1.0) ** j) * zs[j] / np.sqrt(rzs[j]) for j in range(m)], axis=1)
    Y = V @ S[:, :kk]
    Q, kept = orthonormal_basis(Y, drop_rtol)
    return Q, theta[:kk][kept]      # the values of the kept vectors


def arnoldi(apply_B, r0, m, tol=0.0):
    """Basic Arnoldi (Algorithm 1).  Returns (W [n x (j+1)], Hbar [(j+1) x j], beta,
    gmres_rel) after j <= m steps."""
    r0 = np.asarray(r0, dtype=np.float64)
    beta = np.linalg.norm(r0)
    W = [r0 / beta]
    H = np.zeros((m + 1, m))
    rel = 1.0
    j = 0
    while j < m:
        v = apply_B(W[j])
        Wm = np.stack(W, axis=1)
        h = Wm.T @ v
        v = v - Wm @ h
        h2 = Wm.T @ v
        v = v - Wm @ h2
        H[: j + 1, j] = h + h2
        H[j + 1, j] = np.linalg.norm(v)
        j += 1
        e1 = np.zeros(j + 1)
        e1[0] = beta
        y = np.linalg.lstsq(H[: j + 1, :j], e1, rcond=None)[0]
        rel = np.linalg.norm(e1 - H[: j + 1, :j] @ y) / beta
        if H[j, j - 1] == 0.0 or rel <= tol:
            W.append(v / H[j, j - 1] if H[j, j - 1] != 0.0 else np.zeros_like(v))
            break
        W.append(v / H[j, j - 1])
    return np.stack(W, axis=1), H[: j + 1, :j], beta, rel


def arnoldi_coarse_space(W, H, k, eps_tol, drop_rtol=1e-10):
    """Ritz selection from an Arnoldi run (App. A, Eq. A.4; selection |Re lambda| < eps_tol
    of Sec. 5; reading R17).  Returns (Z with orthonormal columns, the selected Ritz
    values)."""
    j = H.shape[1]
    lam, V = np.linalg.eig(H[:j, :j])
    order = np.argsort(lam.real, kind="stable")
    cols, vals = [], []
    taken = np.zeros(j, dtype=bool)
    for i in order:
        if taken[i] or not abs(lam[i].real) < eps_tol or len(vals) >= k:
            continue
        y = W[:, :j] @ V[:, i]
        taken[i] = True
        if abs(lam[i].imag) <= 1e-12 * abs(lam[i]):
            cols.append(y.real)
            vals.append(lam[i].real)
        else:
            cols += [y.real, y.imag]
            vals += [lam[i].real, lam[i].real]
            pair = np.argmin(np.abs(lam - np.conj(lam[i])) + taken * np.inf)
            taken[pair] = True
    if not cols:
        raise ValueError("no Ritz value below eps_tol")
    Y = np.stack(cols, axis=1)
    Q, kept = orthonormal_basis(Y, drop_rtol)
    return Q, np.asarray(vals)[kept]      # the values of the kept vectors


def deflation_apriori(prob):
    """Z_S of Eq. 16-17 (the a priori coarse space of Sec. 3.3.1): column j = fraction
    of each pixel's hits inside interval j, Q/U rows zero; each T row sums to 1."""
    K = prob.offsets.size - 1
    nc = prob.ncomp
    Z = np.zeros((prob.n, K), dtype=np.float64)
    for j in range(K):
        a, b = int(prob.offsets[j]), int(prob.offsets[j + 1])
        pc = prob.pix_c[a:b]
        pc = pc[pc >= 0]
        cnt = np.bincount(pc, minlength=prob.npix_obs).astype(np.float64)
        Z[0::nc, j] = cnt / prob.hits
    return Z


def deflation_apriori_merged(prob, r):
    """Z_S with its K interval columns combined into r groups (Sec. 3.3.1: the column
    count may be reduced by merging stationary periods, keeping every nonzero row's sum
    at 1).  Groups are runs of consecutive intervals: interval i joins group
    floor(i r / K); a merged column is the sum of its members' columns."""
    Z = deflation_apriori(prob)
    K = Z.shape[1]
    if not 1 <= r <= K:
        raise ValueError("need 1 <= r <= K")
    G = np.zeros((K, r), dtype=np.float64)
    G[np.arange(K), (np.arange(K) * r) // K] = 1.0
    return Z @ G


def independent_columns(Z, drop_rtol=DROP_RTOL):
    """Reading R16.  Columns of Z in order, skipping each column whose component
    orthogonal to the kept ones (Gram-Schmidt, projected twice) has norm below drop_rtol
    times the largest column norm of Z (or is zero): Z_S has dependent columns whenever
    intervals see the same hit fractions, Ritz vectors can repeat, and E = Z^T A Z must
    be invertible (Eq. 12).  Returns (the kept columns, their indices)."""
    Z = np.asarray(Z, dtype=np.float64)
    scale = np.linalg.norm(Z, axis=0).max() if Z.shape[1] else 0.0
    Q = np.zeros((Z.shape[0], 0))
    kept = []
    for j in range(Z.shape[1]):
        v = Z[:, j].copy()
        for _ in range(2):
            v -= Q @ (Q.T @ v)
        piv = np.linalg.norm(v)
        if not piv > 0.0 or piv < drop_rtol * scale:
            continue
        kept.append(j)
        Q = np.column_stack([Q, v / piv])
    return Z[:, kept], kept


def orthonormal_basis(Y, drop_rtol=DROP_RTOL):
    """Orthonormal basis of the columns of Y kept by independent_columns (reading R16),
    by Householder QR of the kept columns (np.linalg.qr).  Returns (Q, kept indices)."""
    Yk, kept = independent_columns(Y, drop_rtol)
    if not kept:
        raise ValueError("every column is dependent")
    Q, _ = np.linalg.qr(Yk)
    return Q, kept


__all__ = ["BlockJacobi", "TwoLevel", "lanczos_tridiagonal", "ritz_coarse_space",
           "arnoldi", "arnoldi_coarse_space", "deflation_apriori", "deflation_apriori_merged",
           "independent_columns", "orthonormal_basis"]

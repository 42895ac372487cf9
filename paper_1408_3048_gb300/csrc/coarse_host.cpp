// Host FP64 dense helpers for the a posteriori coarse space (Sec. 3.3.2, App. A):
//   * the k smallest eigenpairs of the symmetric tridiagonal Lanczos matrix T_m, by
//     Sturm-sequence bisection (eigenvalues) and inverse iteration with
//     re-orthogonalisation inside clusters (eigenvectors);
//   * the Cholesky factor and inverses of the coarse operator E = Z^T A Z (App. C).
#include <algorithm>
#include <cmath>

#include "coarse_host.h"

namespace mm {

// number of eigenvalues of T (diag d, off-diag e) strictly smaller than x
static int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
    const int m = (int)d.size();
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < m; ++i) {
        if (q == 0.0) q = 1e-300;
        q = d[i] - x - e[i - 1] * e[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

void tridiag_smallest(const std::vector<double>& d, const std::vector<double>& e, int k,
                      std::vector<double>& theta, std::vector<double>& S) {
    const int m = (int)d.size();
    k = std::min(k, m);
    // Gershgorin bounds
    double lo = d[0], hi = d[0];
    for (int i = 0; i < m; ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    const double scale = std::max(std::fabs(lo), std::fabs(hi));
    theta.assign(k, 0.0);
    for (int j = 0; j < k; ++j) {
        double a = lo, b = hi;   // count(a) <= j < count(b)
        for (int it = 0; it < 200; ++it) {
            const double c = 0.5 * (a + b);
            if (c <= a || c >= b) break;
            if (sturm_count(d, e, c) > j) b = c; else a = c;
            if (b - a <= 4e-16 * scale) break;
        }
        theta[j] = 0.5 * (a + b);
    }
    // inverse iteration: (T - mu I) x = y by Gaussian elimination with partial pivoting
    S.assign((size_t)m * k, 0.0);
    const double eps = 2.2e-16 * scale;
    for (int j = 0; j < k; ++j) {
        const double mu = theta[j] + eps * 0.5;
        std::vector<double> x(m);
        uint64_t st = 0x9E3779B97F4A7C15ull ^ (uint64_t)(j + 1) * 0xBF58476D1CE4E5B9ull;
        for (int i = 0; i < m; ++i) {
            st ^= st >> 31; st *= 0x94D049BB133111EBull; st ^= st >> 29;
            x[i] = ((double)(st >> 11) / 9007199254740992.0) - 0.5;
        }
        for (int iter = 0; iter < 4; ++iter) {
            // tridiagonal LU with pivoting: rows carry (a, b, c) band + fill
            std::vector<double> dd(m), du(m, 0.0), du2(m, 0.0), dl(m, 0.0), rhs = x;
            std::vector<int> piv(m, 0);
            for (int i = 0; i < m; ++i) dd[i] = d[i] - mu;
            for (int i = 0; i + 1 < m; ++i) {
                du[i] = e[i];
                dl[i] = e[i];
            }
            for (int i = 0; i + 1 < m; ++i) {
                if (std::fabs(dd[i]) >= std::fabs(dl[i])) {
                    if (dd[i] == 0.0) dd[i] = eps;
                    const double f = dl[i] / dd[i];
                    dl[i] = f;
                    dd[i + 1] -= f * du[i];
                    piv[i] = 0;
                } else {
                    const double f = dd[i] / dl[i];
                    dd[i] = dl[i];
                    dl[i] = f;
                    const double t = du[i];
                    du[i] = dd[i + 1];
                    dd[i + 1] = t - f * dd[i + 1];
                    if (i + 2 < m) {
                        du2[i] = du[i + 1];
                        du[i + 1] = -f * du[i + 1];
                    }
                    piv[i] = 1;
                }
            }
            if (dd[m - 1] == 0.0) dd[m - 1] = eps;
            // forward: apply L^-1
            for (int i = 0; i + 1 < m; ++i) {
                if (piv[i] == 0) {
                    rhs[i + 1] -= dl[i] * rhs[i];
                } else {
                    const double t = rhs[i];
                    rhs[i] = rhs[i + 1];
                    rhs[i + 1] = t - dl[i] * rhs[i + 1];
                }
            }
            // backward: U x = rhs
            for (int i = m - 1; i >= 0; --i) {
                double v = rhs[i];
                if (i + 1 < m) v -= du[i] * rhs[i + 1];
                if (i + 2 < m) v -= du2[i] * rhs[i + 2];
                rhs[i] = v / dd[i];
            }
            // re-orthogonalise against earlier vectors of the same cluster
            for (int jj = 0; jj < j; ++jj) {
                if (std::fabs(theta[jj] - theta[j]) > 1e-3 * scale) continue;
                double dot = 0.0;
                for (int i = 0; i < m; ++i) dot += rhs[i] * S[(size_t)i * k + jj];
                for (int i = 0; i < m; ++i) rhs[i] -= dot * S[(size_t)i * k + jj];
            }
            double nrm = 0.0;
            for (int i = 0; i < m; ++i) nrm += rhs[i] * rhs[i];
            nrm = std::sqrt(nrm);
            if (!(nrm > 0.0)) break;
            for (int i = 0; i < m; ++i) x[i] = rhs[i] / nrm;
        }
        for (int i = 0; i < m; ++i) S[(size_t)i * k + j] = x[i];
    }
}

// Plain Cholesky E = L L^T (row-major lower); false when E is not positive definite.
bool cholesky_lower(const std::vector<double>& E, int k, std::vector<double>& L) {
    L.assign((size_t)k * k, 0.0);
    for (int j = 0; j < k; ++j) {
        double s = E[(size_t)j * k + j];
        for (int p = 0; p < j; ++p) s -= L[(size_t)j * k + p] * L[(size_t)j * k + p];
        if (!(s > 0.0)) return false;
        const double ljj = std::sqrt(s);
        L[(size_t)j * k + j] = ljj;
        for (int i = j + 1; i < k; ++i) {
            double v = E[(size_t)i * k + j];
            for (int p = 0; p < j; ++p) v -= L[(size_t)i * k + p] * L[(size_t)j * k + p];
            L[(size_t)i * k + j] = v / ljj;
        }
    }
    return true;
}

std::vector<double> spd_inverse_from_cholesky(const std::vector<double>& L, int k) {
    // Y = L^-1 by forward substitution on the identity (lower triangular), E^-1 = Y^T Y
    std::vector<double> Y((size_t)k * k, 0.0);
    for (int c = 0; c < k; ++c) {
        for (int i = c; i < k; ++i) {
            double v = i == c ? 1.0 : 0.0;
            for (int j = c; j < i; ++j) v -= L[(size_t)i * k + j] * Y[(size_t)j * k + c];
            Y[(size_t)i * k + c] = v / L[(size_t)i * k + i];
        }
    }
    std::vector<double> inv((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = 0.0;
            for (int m = std::max(i, j); m < k; ++m) v += Y[(size_t)m * k + i] * Y[(size_t)m * k + j];
            inv[(size_t)i * k + j] = inv[(size_t)j * k + i] = v;
        }
    return inv;
}

using cplx = std::complex<double>;

// Givens rotation (c real, s complex) with [c s; -conj(s) c] [a; b] = [r; 0].
static void givens(cplx a, cplx b, double& c, cplx& s) {
    const double na = std::abs(a), nb = std::abs(b);
    if (nb == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    if (na == 0.0) {
        c = 0.0;
        s = std::conj(b) / nb;
        return;
    }
    const double r = std::hypot(na, nb);
    c = na / r;
    s = (a / na) * std::conj(b) / r;
}

bool hessenberg_eigenvalues(const std::vector<double>& Hin, int n, std::vector<cplx>& lam) {
    std::vector<cplx> A((size_t)n * n);
    for (size_t i = 0; i < A.size(); ++i) A[i] = Hin[i];
    auto at = [&](int i, int j) -> cplx& { return A[(size_t)i * n + j]; };
    lam.assign((size_t)n, cplx(0.0));
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, sweeps = 0;
    std::vector<double> cs((size_t)n);
    std::vector<cplx> sn((size_t)n);
    while (hi >= 0) {
        if (hi == 0) {
            lam[0] = at(0, 0);
            break;
        }
        // start of the unreduced block ending at hi
        int l = hi;
        while (l > 0) {
            const double scale = std::abs(at(l, l)) + std::abs(at(l - 1, l - 1));
            if (std::abs(at(l, l - 1)) <= eps * (scale > 0.0 ? scale : 1.0)) {
                at(l, l - 1) = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {
            lam[(size_t)hi] = at(hi, hi);
            --hi;
            sweeps = 0;
            continue;
        }
        if (++sweeps > 60) return false;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer its last
        // diagonal entry; every 11th sweep an exceptional shift breaks cycles
        cplx mu;
        const cplx a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1), d = at(hi, hi);
        if (sweeps % 11 == 0) {
            mu = d + cplx(std::abs(c), 0.0);
        } else {
            const cplx half = 0.5 * (a + d);
            const cplx disc = std::sqrt(0.25 * (a - d) * (a - d) + b * c);
            const cplx m1 = half + disc, m2 = half - disc;
            mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        }
        // one QR step on rows / columns l..hi: A - mu I = Q R, A <- R Q + mu I
        for (int k = l; k <= hi; ++k) at(k, k) -= mu;
        for (int k = l; k < hi; ++k) {
            double ck;
            cplx sk;
            givens(at(k, k), at(k + 1, k), ck, sk);
            cs[(size_t)k] = ck;
            sn[(size_t)k] = sk;
            for (int j = k; j <= hi; ++j) {
                const cplx x = at(k, j), y = at(k + 1, j);
                at(k, j) = ck * x + sk * y;
                at(k + 1, j) = -std::conj(sk) * x + ck * y;
            }
        }
        for (int k = l; k < hi; ++k) {
            const double ck = cs[(size_t)k];
            const cplx sk = sn[(size_t)k];
            const int top = std::min(k + 2, hi);
            for (int i = l; i <= top; ++i) {
                const cplx x = at(i, k), y = at(i, k + 1);
                at(i, k) = ck * x + std::conj(sk) * y;
                at(i, k + 1) = -sk * x + ck * y;
            }
        }
        for (int k = l; k <= hi; ++k) at(k, k) += mu;
    }
    return true;
}

std::vector<cplx> hessenberg_eigenvector(const std::vector<double>& Hin, int n, cplx lam) {
    double hnorm = 0.0;
    for (double v : Hin) hnorm = std::max(hnorm, std::abs(v));
    // a tiny offset keeps H - lam I invertible when lam is exact to rounding
    const cplx shift = lam + cplx(1e-13 * (hnorm > 0.0 ? hnorm : 1.0), 0.0);
    std::vector<cplx> U((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) U[(size_t)i * n + j] = Hin[(size_t)i * n + j] - (i == j ? shift : cplx(0.0));
    // Hessenberg LU with partial pivoting between neighbouring rows: P_k L_k records
    std::vector<cplx> mult((size_t)n, cplx(0.0));
    std::vector<char> swapped((size_t)n, 0);
    for (int k = 0; k + 1 < n; ++k) {
        cplx* r0 = &U[(size_t)k * n];
        cplx* r1 = &U[(size_t)(k + 1) * n];
        if (std::abs(r1[k]) > std::abs(r0[k])) {
            for (int j = k; j < n; ++j) std::swap(r0[j], r1[j]);
            swapped[(size_t)k] = 1;
        }
        const cplx m = r0[k] != cplx(0.0) ? r1[k] / r0[k] : cplx(0.0);
        mult[(size_t)k] = m;
        for (int j = k; j < n; ++j) r1[j] -= m * r0[j];
    }
    for (int i = 0; i < n; ++i)
        if (U[(size_t)i * n + i] == cplx(0.0)) U[(size_t)i * n + i] = cplx(1e-300, 0.0);
    std::vector<cplx> x((size_t)n, cplx(1.0, 0.0));
    for (int it = 0; it < 3; ++it) {
        // apply the row operations to the right-hand side, then back substitution
        for (int k = 0; k + 1 < n; ++k) {
            if (swapped[(size_t)k]) std::swap(x[(size_t)k], x[(size_t)k + 1]);
            x[(size_t)k + 1] -= mult[(size_t)k] * x[(size_t)k];
        }
        for (int i = n - 1; i >= 0; --i) {
            cplx v = x[(size_t)i];
            for (int j = i + 1; j < n; ++j) v -= U[(size_t)i * n + j] * x[(size_t)j];
            x[(size_t)i] = v / U[(size_t)i * n + i];
        }
        double nrm = 0.0;
        for (const cplx& v : x) nrm += std::norm(v);
        nrm = std::sqrt(nrm);
        for (cplx& v : x) v /= nrm;
    }
    return x;
}

bool lu_inverse(const std::vector<double>& E, int k, std::vector<double>& inv, double* min_pivot_ratio) {
    // Gauss-Jordan on [E | I] with partial pivoting (the LU route of App. C)
    std::vector<double> a(E);
    inv.assign((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) inv[(size_t)i * k + i] = 1.0;
    double maxabs = 0.0;
    for (double v : E) maxabs = std::max(maxabs, std::fabs(v));
    double minpiv = 1e300;
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (std::fabs(a[(size_t)r * k + c]) > std::fabs(a[(size_t)p * k + c])) p = r;
        const double piv = a[(size_t)p * k + c];
        minpiv = std::min(minpiv, std::fabs(piv));
        if (piv == 0.0) return false;
        if (p != c) {
            for (int j = 0; j < k; ++j) {
                std::swap(a[(size_t)p * k + j], a[(size_t)c * k + j]);
                std::swap(inv[(size_t)p * k + j], inv[(size_t)c * k + j]);
            }
        }
        for (int j = 0; j < k; ++j) {
            a[(size_t)c * k + j] /= piv;
            inv[(size_t)c * k + j] /= piv;
        }
        for (int r = 0; r < k; ++r) {
            if (r == c) continue;
            const double f = a[(size_t)r * k + c];
            if (f == 0.0) continue;
            for (int j = 0; j < k; ++j) {
                a[(size_t)r * k + j] -= f * a[(size_t)c * k + j];
                inv[(size_t)r * k + j] -= f * inv[(size_t)c * k + j];
            }
        }
    }
    if (min_pivot_ratio) *min_pivot_ratio = maxabs > 0.0 ? minpiv / maxabs : 0.0;
    return true;
}

}  // namespace mm

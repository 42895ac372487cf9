// Host FP64 dense helpers of the coarse-space construction (see coarse_host.cpp).
#pragma once

#include <stdint.h>

#include <complex>
#include <vector>

namespace mm {

// k smallest eigenpairs of the symmetric tridiagonal matrix (diag d[m], off-diag e[m-1]):
// theta[k] ascending, S row-major m x k (unit eigenvectors).
void tridiag_smallest(const std::vector<double>& d, const std::vector<double>& e, int k,
                      std::vector<double>& theta, std::vector<double>& S);

// E = L L^T, row-major lower L; false if E is not positive definite.
bool cholesky_lower(const std::vector<double>& E, int k, std::vector<double>& L);
// E^-1 (row-major, symmetric) from the lower Cholesky factor L of E: L^-T L^-1.
std::vector<double> spd_inverse_from_cholesky(const std::vector<double>& L, int k);

// E^-1 by Gauss-Jordan elimination with partial pivoting; false on an exactly zero
// pivot.  *min_pivot_ratio (may be null) = smallest |pivot| / max |E_ij|.
bool lu_inverse(const std::vector<double>& E, int k, std::vector<double>& inv, double* min_pivot_ratio);

// Eigenvalues of a real upper Hessenberg matrix H (row-major n x n) by the shifted QR
// algorithm in complex arithmetic (Givens rotations, Wilkinson shifts, deflation on
// negligible subdiagonals); false if an eigenvalue needs more than 60 sweeps.
bool hessenberg_eigenvalues(const std::vector<double>& H, int n, std::vector<std::complex<double>>& lam);

// Unit eigenvector of H for the (computed) eigenvalue lam by inverse iteration with a
// pivoted Hessenberg LU of H - lam I (O(n^2) per solve).
std::vector<std::complex<double>> hessenberg_eigenvector(const std::vector<double>& H, int n,
                                                         std::complex<double> lam);

}  // namespace mm

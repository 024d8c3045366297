// Small dense complex linear algebra on the host (Rayleigh-Ritz of the deflation set-up).
#pragma once

#include <complex>
#include <vector>

namespace sgn {

// Eigen-decomposition of a general complex n x n matrix G (row-major):
// w = eigenvalues, X = unit-norm eigenvectors as columns (row-major n x n).
// Returns 0 on success, 1 if the QR iteration did not converge.
int dense_eig(int n, const std::vector<std::complex<double>>& G, std::vector<std::complex<double>>& w,
              std::vector<std::complex<double>>& X, int max_iter = 60);

// Hermitian G: eigenvalues (real parts of the Schur diagonal) and the unitary
// Schur vectors, which are the orthonormal eigenvectors.  Returns 1 on failure.
int herm_eig(int n, const std::vector<std::complex<double>>& G, std::vector<double>& w,
             std::vector<std::complex<double>>& X);

// Solve A X = B (A n x n, B n x r, both row-major) in place of B.  Returns 1 if singular.
int dense_solve(int n, int r, std::vector<std::complex<double>> A, std::vector<std::complex<double>>& B);

// Upper Cholesky factor R of a Hermitian positive definite G = R^dag R.  Returns 1 if not HPD.
int cholesky_upper(int n, const std::vector<std::complex<double>>& G, std::vector<std::complex<double>>& R);

}  // namespace sgn

// Small dense complex FP64 linear algebra on the host, for the per-cycle problems of the Krylov
// solvers (least squares with the (m+1) x m Hessenberg matrix, harmonic Ritz eigenproblems,
// Rayleigh-Ritz).  Sizes are at most a few hundred, so plain O(n^3) algorithms suffice.
#pragma once

#include <complex>
#include <vector>

namespace dense {

using cd = std::complex<double>;

// column-major matrix
struct Mat {
  int r = 0, c = 0;
  std::vector<cd> a;
  Mat() = default;
  Mat(int rows, int cols) : r(rows), c(cols), a((size_t)rows * cols, cd(0.0, 0.0)) {}
  cd &operator()(int i, int j) { return a[(size_t)j * r + i]; }
  const cd &operator()(int i, int j) const { return a[(size_t)j * r + i]; }
};

Mat matmul(const Mat &A, const Mat &B);
Mat adjoint(const Mat &A);

// d = argmin || c - A d ||_2 (A: rows >= cols, full column rank) by Householder QR
std::vector<cd> lstsq(const Mat &A, const std::vector<cd> &c);

// The same in two steps, for many right-hand sides c with one A: the Householder factorisation
// once (R in the upper triangle of `a`, the reflections in v / beta), then per c the reflections and
// the back substitution (bit-identical to lstsq)
struct QRFact {
  Mat a;
  std::vector<std::vector<cd>> v;
  std::vector<double> beta;
};
QRFact qr_factor(const Mat &A);
std::vector<cd> qr_solve(const QRFact &f, const std::vector<cd> &c);

// x = A^{-1} b by LU with partial pivoting; returns false on an exactly zero pivot
bool solve(const Mat &A, const std::vector<cd> &b, std::vector<cd> &x);

// Complex Schur decomposition A = Z T Z^H (Hessenberg reduction + shifted QR);
// returns false if the iteration did not converge
bool schur(const Mat &A, Mat &T, Mat &Z);

// eigenvalues w and unit-norm right eigenvectors X (columns) of a general complex matrix
bool eig(const Mat &A, std::vector<cd> &w, Mat &X);

// Hermitian eigen-decomposition (A is symmetrised first): real w ascending, orthonormal X
bool eigh(const Mat &A, std::vector<double> &w, Mat &X);

// Hermitian-definite generalised problem A g = mu B g (B positive definite): mu ascending,
// G with G^H B G = I
bool eigh_gen(const Mat &A, const Mat &B, std::vector<double> &mu, Mat &G);

// Orthonormalise the columns of A in order (classical Gram-Schmidt applied twice)
Mat orthonormalize(const Mat &A);

}  // namespace dense

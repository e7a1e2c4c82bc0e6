// Plain float64 CPU oracle of randomized block orthogonalization and s-step GMRES
// (Yamazaki, Higgins, Boman and Szyld, arXiv 2503.16717) -- TEST INFRASTRUCTURE ONLY.
//
// Nothing in the library links or loads this code; only the tests (through
// oracle/cpp_oracle.py) call it.  It restates the schemes step by step in the paper's
// order, with plain loops over column-major float64 arrays (no BLAS, no blocking, no
// reordering), and shares no code with the CUDA library.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <stdexcept>
#include <vector>

namespace oracle {

// A column-major m x n float64 matrix.
struct Mat {
  int64_t m = 0, n = 0;
  std::vector<double> a;
  Mat() = default;
  Mat(int64_t rows, int64_t cols) : m(rows), n(cols), a((size_t)(rows * cols), 0.0) {}
  double& operator()(int64_t i, int64_t j) { return a[(size_t)(i + j * m)]; }
  double operator()(int64_t i, int64_t j) const { return a[(size_t)(i + j * m)]; }
  double* col(int64_t j) { return a.data() + j * m; }
  const double* col(int64_t j) const { return a.data() + j * m; }
};

// Columns [j0, j0 + k) of A as a new matrix.
inline Mat cols(const Mat& A, int64_t j0, int64_t k) {
  Mat B(A.m, k);
  for (int64_t j = 0; j < k; ++j)
    for (int64_t i = 0; i < A.m; ++i) B(i, j) = A(i, j0 + j);
  return B;
}

// A Cholesky factorisation met a non-positive (or non-finite) pivot (Section 5.1).
struct Breakdown {
  int column;
  const char* where;
};

// ---- sketch.cpp -------------------------------------------------------------------------
uint64_t splitmix64_output(uint64_t seed, uint64_t i);
// Indices (nrows x zeta, row-major) and signs of the sparse-sign sketch's columns
// row0 .. row0 + nrows - 1; returns false when a row found fewer than zeta distinct
// indices in 64 draws.
bool sparse_sign_entries(int64_t row0, int64_t nrows, int d, int zeta, uint64_t seed,
                         int32_t* idx, int8_t* sgn);
// The sketch as a functor: S W for W with n rows.
struct Sketch {
  int64_t n = 0;
  int d = 0, zeta = 0;
  uint64_t seed = 0;
  std::vector<int32_t> idx;
  std::vector<int8_t> sgn;
  Sketch(int64_t n_, int d_, int zeta_, uint64_t seed_);
  Mat apply(const Mat& W) const;
};
double gaussian_entry(uint64_t seed, uint64_t r, int k, int d);

// ---- dense.cpp --------------------------------------------------------------------------
// G = R^T R, R upper triangular; returns -1 or the first column whose pivot is not
// positive / not finite (R then valid above it).
int cholesky_upper(const Mat& G, Mat& R);
// Householder QR of an m x k matrix (m >= k): R with a non-negative diagonal, and the
// thin Q when want_q.
void householder_qr(const Mat& A, Mat& R, Mat* Q);
// X = W R^{-1} for upper-triangular R.
Mat solve_right_upper(const Mat& W, const Mat& R);
// C = X^T Y with products and sums in long double.
Mat gram(const Mat& X, const Mat& Y);
Mat matmul(const Mat& A, const Mat& B);            // A B
Mat matmul_tn(const Mat& A, const Mat& B);         // A^T B (float64 sums, column order)
Mat sub(const Mat& A, const Mat& B);               // A - B
Mat add(const Mat& A, const Mat& B);               // A + B

// ---- metrics.cpp ------------------------------------------------------------------------
// Eigenvalues of a symmetric k x k matrix (cyclic Jacobi rotations).
std::vector<double> sym_eigenvalues(Mat S);
double orth_error(const Mat& Q);                      // ||I - Q^T Q||_2   (eq. (1))
double backward_error(const Mat& V, const Mat& Q, const Mat& R);  // ||V - QR||_2/||V||_2 (eq. (2))

}  // namespace oracle

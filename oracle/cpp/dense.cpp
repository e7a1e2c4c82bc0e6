// Small dense kernels of the oracle (test infrastructure).
//   * cholesky_upper: G = R^T R column by column; the first pivot that is not positive
//     (or not finite) is the breakdown of CholQR that Section 5.1 and the caption of
//     Figure 4 describe ("non-positive pivots");
//   * householder_qr: Householder QR (Golub and Van Loan, Algorithm 5.2.1) written out,
//     R with a non-negative diagonal (the normalisation in the caption of Figure 1);
//   * solve_right_upper: X = W R^{-1}, the triangular solve of CholQR and RandHH;
//   * gram: C = X^T Y, the reduction of BCGS and CholQR (Section 9), in long double.
#include "common.hpp"

namespace oracle {

int cholesky_upper(const Mat& G, Mat& R) {
  const int64_t k = G.n;
  R = Mat(k, k);
  for (int64_t j = 0; j < k; ++j) {
    double piv = G(j, j);
    for (int64_t i = 0; i < j; ++i) piv -= R(i, j) * R(i, j);
    if (!std::isfinite(piv) || piv <= 0.0) return (int)j;
    const double rjj = std::sqrt(piv);
    R(j, j) = rjj;
    for (int64_t c = j + 1; c < k; ++c) {
      double v = G(j, c);
      for (int64_t i = 0; i < j; ++i) v -= R(i, j) * R(i, c);
      R(j, c) = v / rjj;
    }
  }
  return -1;
}

void householder_qr(const Mat& Ain, Mat& R, Mat* Q) {
  Mat A = Ain;
  const int64_t m = A.m, k = A.n;
  if (m < k) throw std::runtime_error("householder_qr needs m >= k");
  std::vector<std::vector<double>> vs((size_t)k);
  std::vector<double> betas((size_t)k, 0.0);
  for (int64_t j = 0; j < k; ++j) {
    double ss = 0.0;
    for (int64_t i = j; i < m; ++i) ss += A(i, j) * A(i, j);
    const double alpha = std::sqrt(ss);
    if (alpha == 0.0) continue;
    // reflect x onto -sign(x0) alpha e1 (no cancellation in v0)
    std::vector<double> v((size_t)(m - j));
    for (int64_t i = j; i < m; ++i) v[(size_t)(i - j)] = A(i, j);
    const double s = v[0] >= 0.0 ? 1.0 : -1.0;
    v[0] += s * alpha;
    double vv = 0.0;
    for (double x : v) vv += x * x;
    const double beta = 2.0 / vv;
    for (int64_t c = j; c < k; ++c) {
      double w = 0.0;
      for (int64_t i = j; i < m; ++i) w += v[(size_t)(i - j)] * A(i, c);
      for (int64_t i = j; i < m; ++i) A(i, c) -= beta * v[(size_t)(i - j)] * w;
    }
    vs[(size_t)j] = v;
    betas[(size_t)j] = beta;
  }
  R = Mat(k, k);
  std::vector<double> sgn((size_t)k);
  for (int64_t i = 0; i < k; ++i) sgn[(size_t)i] = A(i, i) < 0.0 ? -1.0 : 1.0;
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i <= c; ++i) R(i, c) = sgn[(size_t)i] * A(i, c);
  if (!Q) return;
  Mat QQ(m, k);
  for (int64_t i = 0; i < k; ++i) QQ(i, i) = 1.0;
  for (int64_t j = k - 1; j >= 0; --j) {
    const std::vector<double>& v = vs[(size_t)j];
    if (v.empty()) continue;
    for (int64_t c = 0; c < k; ++c) {
      double w = 0.0;
      for (int64_t i = j; i < m; ++i) w += v[(size_t)(i - j)] * QQ(i, c);
      for (int64_t i = j; i < m; ++i) QQ(i, c) -= betas[(size_t)j] * v[(size_t)(i - j)] * w;
    }
  }
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < m; ++i) QQ(i, c) *= sgn[(size_t)c];
  *Q = QQ;
}

// X R = W: each row x of X solves x R = w by substitution over the columns.
Mat solve_right_upper(const Mat& W, const Mat& R) {
  Mat X(W.m, W.n);
  for (int64_t r = 0; r < W.m; ++r)
    for (int64_t j = 0; j < W.n; ++j) {
      double v = W(r, j);
      for (int64_t l = 0; l < j; ++l) v -= X(r, l) * R(l, j);
      X(r, j) = v / R(j, j);
    }
  return X;
}

Mat gram(const Mat& X, const Mat& Y) {
  Mat C(X.n, Y.n);
  for (int64_t i = 0; i < X.n; ++i)
    for (int64_t j = 0; j < Y.n; ++j) {
      long double s = 0.0L;
      for (int64_t r = 0; r < X.m; ++r) s += (long double)X(r, i) * (long double)Y(r, j);
      C(i, j) = (double)s;
    }
  return C;
}

Mat matmul(const Mat& A, const Mat& B) {
  Mat C(A.m, B.n);
  for (int64_t j = 0; j < B.n; ++j)
    for (int64_t l = 0; l < A.n; ++l) {
      const double b = B(l, j);
      for (int64_t i = 0; i < A.m; ++i) C(i, j) += A(i, l) * b;
    }
  return C;
}

Mat matmul_tn(const Mat& A, const Mat& B) {
  Mat C(A.n, B.n);
  for (int64_t i = 0; i < A.n; ++i)
    for (int64_t j = 0; j < B.n; ++j) {
      double s = 0.0;
      for (int64_t r = 0; r < A.m; ++r) s += A(r, i) * B(r, j);
      C(i, j) = s;
    }
  return C;
}

Mat sub(const Mat& A, const Mat& B) {
  Mat C = A;
  for (size_t t = 0; t < C.a.size(); ++t) C.a[t] -= B.a[t];
  return C;
}

Mat add(const Mat& A, const Mat& B) {
  Mat C = A;
  for (size_t t = 0; t < C.a.size(); ++t) C.a[t] += B.a[t];
  return C;
}

}  // namespace oracle

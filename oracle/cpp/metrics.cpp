// Accuracy measures of a computed QR factorisation (oracle; test infrastructure):
//   ||I - Q^T Q||_2 (equation (1), Section 4) and ||V - Q R||_2 / ||V||_2 (equation
//   (2)), with the products in long double; the 2-norms from the eigenvalues of small
//   symmetric matrices by the cyclic Jacobi method (Golub and Van Loan, Section 8.5).
#include "common.hpp"

namespace oracle {

std::vector<double> sym_eigenvalues(Mat S) {
  const int64_t k = S.n;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int64_t j = 0; j < k; ++j)
      for (int64_t i = 0; i < k; ++i) {
        tot += S(i, j) * S(i, j);
        if (i != j) off += S(i, j) * S(i, j);
      }
    if (off <= 1e-34 * tot || off == 0.0) break;
    for (int64_t p = 0; p < k; ++p)
      for (int64_t q = p + 1; q < k; ++q) {
        const double apq = S(p, q);
        if (apq == 0.0) continue;
        // the rotation that zeroes S(p, q): t = tan of its angle, the smaller root
        const double theta = (S(q, q) - S(p, p)) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int64_t r = 0; r < k; ++r) {  // columns p, q
          const double sp = S(r, p), sq = S(r, q);
          S(r, p) = c * sp - s * sq;
          S(r, q) = s * sp + c * sq;
        }
        for (int64_t r = 0; r < k; ++r) {  // rows p, q
          const double sp = S(p, r), sq = S(q, r);
          S(p, r) = c * sp - s * sq;
          S(q, r) = s * sp + c * sq;
        }
      }
  }
  std::vector<double> ev((size_t)k);
  for (int64_t i = 0; i < k; ++i) ev[(size_t)i] = S(i, i);
  return ev;
}

static double max_abs(const std::vector<double>& v) {
  double m = 0.0;
  for (double x : v) m = std::fmax(m, std::fabs(x));
  return m;
}

double orth_error(const Mat& Q) {
  const int64_t c = Q.n;
  if (c == 0) return 0.0;
  Mat E(c, c);
  for (int64_t i = 0; i < c; ++i)
    for (int64_t j = 0; j < c; ++j) {
      long double s = (i == j) ? 1.0L : 0.0L;
      for (int64_t r = 0; r < Q.m; ++r) s -= (long double)Q(r, i) * (long double)Q(r, j);
      E(i, j) = (double)s;
    }
  Mat Es(c, c);
  for (int64_t i = 0; i < c; ++i)
    for (int64_t j = 0; j < c; ++j) Es(i, j) = 0.5 * (E(i, j) + E(j, i));
  return max_abs(sym_eigenvalues(Es));
}

// ||A||_2 of a tall matrix held in long double: sqrt of the largest eigenvalue of A^T A
static double norm2_tall(const std::vector<long double>& A, int64_t m, int64_t c) {
  Mat G(c, c);
  for (int64_t i = 0; i < c; ++i)
    for (int64_t j = 0; j < c; ++j) {
      long double s = 0.0L;
      for (int64_t r = 0; r < m; ++r) s += A[(size_t)(r + i * m)] * A[(size_t)(r + j * m)];
      G(i, j) = (double)s;
    }
  return std::sqrt(std::fmax(0.0, max_abs(sym_eigenvalues(G))));
}

double backward_error(const Mat& V, const Mat& Q, const Mat& R) {
  const int64_t m = V.m, c = V.n;
  std::vector<long double> D((size_t)(m * c)), Vl((size_t)(m * c));
  for (int64_t j = 0; j < c; ++j)
    for (int64_t r = 0; r < m; ++r) {
      long double s = (long double)V(r, j);
      for (int64_t l = 0; l < Q.n; ++l) s -= (long double)Q(r, l) * (long double)R(l, j);
      // the difference is rounded to float64 before its norm is taken
      D[(size_t)(r + j * m)] = (long double)(double)s;
      Vl[(size_t)(r + j * m)] = (long double)V(r, j);
    }
  const double nv = norm2_tall(Vl, m, c);
  const double nd = norm2_tall(D, m, c);
  return nv > 0.0 ? nd / nv : nd;
}

}  // namespace oracle

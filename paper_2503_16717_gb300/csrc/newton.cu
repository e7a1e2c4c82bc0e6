// Parameters of the Newton and Chebyshev matrix-powers bases (host code), both as the
// real three-term recurrence
//   v_{i+1} = (A - alpha_i) v_i + beta_i v_{i-1}.
// Newton: the Ritz values of the Hessenberg matrix of a GMRES cycle in the modified
// Leja ordering of Bai, Hu and Reichel (IMA J. Numer. Anal. 14, 1994); beta_i =
// (Im theta)^2 for the second value of a conjugate pair, else 0.
// Chebyshev (Joubert and Carey, Comput. Math. Appl. 24, 1992): the scaled Chebyshev
// polynomials 2 (e/2)^k T_k((z - c)/e) of an ellipse with centre c and half focal
// distance e enclosing the Ritz values (e^2 < 0: foci on the line Re z = c).
#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>
#include <vector>

#include "rbo_internal.cuh"

namespace rbo {

// Eigenvalues of the k x k upper Hessenberg matrix A (column-major, ld k; destroyed)
// by the implicitly double-shifted QR algorithm (Francis 1961): the active block is
// split at negligible subdiagonal entries, 1 x 1 and 2 x 2 blocks are read off its
// bottom, otherwise a 3 x 3 bulge started by the first column of (A - s1)(A - s2)
// (s1, s2 the eigenvalues of the trailing 2 x 2 block) is chased down with
// Householder reflectors.  Returns false if a block needs more than 200 sweeps.
static bool hessenberg_eig(std::vector<double>& A, int k, std::vector<double>& wr,
                           std::vector<double>& wi) {
  auto a = [&](int i, int j) -> double& { return A[(size_t)i + (size_t)j * k]; };
  const double eps = std::numeric_limits<double>::epsilon();
  double anorm = 0.0;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i <= std::min(j + 1, k - 1); ++i) anorm = std::max(anorm, std::fabs(a(i, j)));
  if (anorm == 0.0) anorm = 1.0;
  wr.assign(k, 0.0);
  wi.assign(k, 0.0);
  int hi = k - 1, its = 0;
  while (hi >= 0) {
    int lo = hi;
    while (lo > 0) {
      double sc = std::fabs(a(lo - 1, lo - 1)) + std::fabs(a(lo, lo));
      if (sc == 0.0) sc = anorm;
      if (std::fabs(a(lo, lo - 1)) <= eps * sc) {
        a(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      wr[hi] = a(hi, hi);
      --hi;
      its = 0;
      continue;
    }
    if (lo == hi - 1) {
      const double p = a(hi - 1, hi - 1), q = a(hi - 1, hi), r = a(hi, hi - 1), t = a(hi, hi);
      const double half = 0.5 * (p + t), det = p * t - q * r, disc = half * half - det;
      if (disc >= 0.0) {
        const double l1 = half + std::copysign(std::sqrt(disc), half);
        wr[hi - 1] = l1;
        wr[hi] = l1 != 0.0 ? det / l1 : 0.0;
      } else {
        wr[hi - 1] = wr[hi] = half;
        wi[hi - 1] = std::sqrt(-disc);
        wi[hi] = -wi[hi - 1];
      }
      hi -= 2;
      its = 0;
      continue;
    }
    if (++its > 200) return false;
    double tr, det;
    if (its % 11 == 0) {  // exceptional shifts break rare cycles
      const double w = std::fabs(a(hi, hi - 1)) + std::fabs(a(hi - 1, hi - 2));
      tr = 1.5 * w;
      det = w * w;
    } else {
      const double p = a(hi - 1, hi - 1), q = a(hi - 1, hi), r = a(hi, hi - 1), t = a(hi, hi);
      tr = p + t;
      det = p * t - q * r;
    }
    double x = a(lo, lo) * a(lo, lo) + a(lo, lo + 1) * a(lo + 1, lo) - tr * a(lo, lo) + det;
    double y = a(lo + 1, lo) * (a(lo, lo) + a(lo + 1, lo + 1) - tr);
    double z = a(lo + 1, lo) * a(lo + 2, lo + 1);
    for (int m = lo; m <= hi - 1; ++m) {
      const bool three = m <= hi - 2;
      const double nrm = std::sqrt(x * x + y * y + (three ? z * z : 0.0));
      const double alpha = x >= 0.0 ? -nrm : nrm;
      const double v0 = x - alpha, v1 = y, v2 = three ? z : 0.0;
      const double vv = v0 * v0 + v1 * v1 + v2 * v2;
      if (vv != 0.0) {
        const double bt = 2.0 / vv;
        for (int j = std::max(lo, m - 1); j <= hi; ++j) {
          double w = v0 * a(m, j) + v1 * a(m + 1, j);
          if (three) w += v2 * a(m + 2, j);
          w *= bt;
          a(m, j) -= w * v0;
          a(m + 1, j) -= w * v1;
          if (three) a(m + 2, j) -= w * v2;
        }
        for (int i = lo; i <= std::min(m + 3, hi); ++i) {
          double w = a(i, m) * v0 + a(i, m + 1) * v1;
          if (three) w += a(i, m + 2) * v2;
          w *= bt;
          a(i, m) -= w * v0;
          a(i, m + 1) -= w * v1;
          if (three) a(i, m + 2) -= w * v2;
        }
      }
      if (m + 1 <= hi - 1) {
        x = a(m + 1, m);
        y = a(m + 2, m);
        z = (m + 3 <= hi) ? a(m + 3, m) : 0.0;
      }
    }
  }
  return true;
}

// Modified Leja ordering: largest modulus first; then the point maximising the sum of
// log distances to the points chosen so far; a complex point is followed by its
// conjugate.  Values with |Im| <= 1e-12 max|theta| count as real.
static std::vector<std::complex<double>> leja(const std::vector<double>& wr,
                                              const std::vector<double>& wi) {
  double scale = 0.0;
  for (size_t i = 0; i < wr.size(); ++i) scale = std::max(scale, std::hypot(wr[i], wi[i]));
  if (scale == 0.0) scale = 1.0;
  std::vector<std::complex<double>> cand, out;
  for (size_t i = 0; i < wr.size(); ++i) {
    if (std::fabs(wi[i]) <= 1e-12 * scale)
      cand.emplace_back(wr[i], 0.0);
    else if (wi[i] > 0.0)
      cand.emplace_back(wr[i], wi[i]);
  }
  const double tiny = 1e-300 * scale;
  while (!cand.empty()) {
    size_t best = 0;
    double bs = -std::numeric_limits<double>::infinity();
    for (size_t c = 0; c < cand.size(); ++c) {
      double sc;
      if (out.empty()) {
        sc = std::abs(cand[c]);
      } else {
        sc = 0.0;
        for (const auto& w : out) sc += std::log(std::max(std::abs(cand[c] - w), tiny));
      }
      if (sc > bs) {
        bs = sc;
        best = c;
      }
    }
    const std::complex<double> z = cand[best];
    cand.erase(cand.begin() + (long)best);
    out.push_back(z);
    if (z.imag() != 0.0) out.push_back(std::conj(z));
  }
  return out;
}

int newton_shifts(const double* H, int64_t ld, int k, int s, double* alpha, double* beta) {
  if (!H || k < 1 || ld < k || s < 1 || !alpha || !beta) return RBO_ERR_ARG;
  std::vector<double> A((size_t)k * k), wr, wi;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) A[(size_t)i + (size_t)j * k] = (i <= j + 1) ? H[i + j * ld] : 0.0;
  for (int i = 0; i < s; ++i) alpha[i] = beta[i] = 0.0;
  if (!hessenberg_eig(A, k, wr, wi)) return RBO_ERR_NOT_CONVERGED;
  const auto order = leja(wr, wi);
  int i = 0;
  while (i < s && i < (int)order.size()) {
    const auto z = order[(size_t)i];
    alpha[i] = z.real();
    if (z.imag() > 0.0 && i + 1 < s) {
      alpha[i + 1] = z.real();
      beta[i + 1] = z.imag() * z.imag();
      i += 2;
    } else {
      ++i;
    }
  }
  return RBO_OK;
}

// Chebyshev basis: the ellipse has its centre c at the midpoint of the Ritz values'
// real extent and its axes along the real and imaginary directions, and is the one of
// smallest capacity (a + b)/2 that encloses every value.  For a real semi-axis a the
// smallest b is b(a) = max_i y_i a / sqrt(a^2 - dx_i^2) (dx_i = Re theta_i - c,
// y_i = |Im theta_i|); a + b(a) is convex for a above half the real extent a0, so a is
// found by bisection on the sign of the right derivative 1 - y_i dx_i^2 / (a^2 -
// dx_i^2)^(3/2), i the maximising value.  A real spectrum gives its interval (b = 0),
// values on one vertical line the segment (a = 0).  With e2 = a^2 - b^2 the
// recurrence is alpha_i = c, beta_0 = 0, beta_1 = -e2 / 2, beta_i = -e2 / 4 (i >= 2).
static void chebyshev_ellipse(const std::vector<double>& wr, const std::vector<double>& wi,
                              double& c, double& a, double& b) {
  const size_t k = wr.size();
  double xmin = wr[0], xmax = wr[0], b0 = 0.0;
  for (size_t i = 0; i < k; ++i) {
    xmin = std::min(xmin, wr[i]);
    xmax = std::max(xmax, wr[i]);
    b0 = std::max(b0, std::fabs(wi[i]));
  }
  c = 0.5 * (xmax + xmin);
  const double a0 = 0.5 * (xmax - xmin);
  if (b0 == 0.0) {
    a = a0;
    b = 0.0;
    return;
  }
  if (a0 == 0.0) {
    a = 0.0;
    b = b0;
    return;
  }
  std::vector<double> dx, y;
  for (size_t i = 0; i < k; ++i)
    if (wi[i] != 0.0) {
      dx.push_back(wr[i] - c);
      y.push_back(std::fabs(wi[i]));
    }
  // b(a) and the right derivative of a + b(a)
  auto eval = [&](double av, double& slope) -> double {
    double best = -1.0;
    size_t bi = 0;
    for (size_t i = 0; i < dx.size(); ++i) {
      const double g = y[i] * av / std::sqrt(av * av - dx[i] * dx[i]);
      if (g > best) {
        best = g;
        bi = i;
      }
    }
    const double r = av * av - dx[bi] * dx[bi];
    slope = 1.0 - y[bi] * dx[bi] * dx[bi] / (r * std::sqrt(r));
    return best;
  };
  double slope;
  const double a1 = 2.0 * a0 + b0;
  double lo = a0, hi = a1 + eval(a1, slope);  // a* <= a* + b(a*) <= a1 + b(a1)
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    eval(mid, slope);
    if (slope < 0.0)
      lo = mid;
    else
      hi = mid;
  }
  a = hi;
  b = eval(hi, slope);
}

int chebyshev_shifts(const double* H, int64_t ld, int k, int s, double* alpha, double* beta) {
  if (!H || k < 1 || ld < k || s < 1 || !alpha || !beta) return RBO_ERR_ARG;
  std::vector<double> A((size_t)k * k), wr, wi;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) A[(size_t)i + (size_t)j * k] = (i <= j + 1) ? H[i + j * ld] : 0.0;
  for (int i = 0; i < s; ++i) alpha[i] = beta[i] = 0.0;
  if (!hessenberg_eig(A, k, wr, wi)) return RBO_ERR_NOT_CONVERGED;
  double c, a, b;
  chebyshev_ellipse(wr, wi, c, a, b);
  const double e2 = a * a - b * b;
  for (int i = 0; i < s; ++i) {
    alpha[i] = c;
    beta[i] = i == 0 ? 0.0 : (i == 1 ? -0.5 * e2 : -0.25 * e2);
  }
  return RBO_OK;
}

}  // namespace rbo

extern "C" int rbo_chebyshev_shifts(const double* H, int64_t ld, int32_t k, int32_t s, double* alpha,
                                    double* beta) {
  return rbo::chebyshev_shifts(H, ld, k, s, alpha, beta);
}

extern "C" int rbo_newton_shifts(const double* H, int64_t ld, int32_t k, int32_t s, double* alpha,
                                 double* beta) {
  return rbo::newton_shifts(H, ld, k, s, alpha, beta);
}

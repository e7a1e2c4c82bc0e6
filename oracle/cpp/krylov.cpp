// CSR SpMV, monomial matrix-powers kernel and s-step GMRES (oracle; test
// infrastructure).  s-step GMRES (Section 4, Figure 1), right-preconditioned: the
// iteration works on y with x = M^{-1} y and the operator Ahat = A M^{-1}; for the
// Jacobi preconditioner M = diag(A), Ahat is A with its columns divided by the
// diagonal.  Readings of the points the paper leaves open:
//   * start: r = b - Ahat y, beta = ||r||, q_0 = r / beta (the V_0 = [v_0] block);
//   * panel: the matrix-powers kernel applies Ahat s times to the panel's start vector
//     u (monomial basis): one-stage, u is the last orthonormal basis vector; two-stage,
//     u is the last preprocessed vector of the previous panel inside a big panel and
//     the last final basis vector at a big-panel boundary (Section 8);
//   * Hessenberg: with the generators U = Q X (X upper triangular) and the outputs
//     W = Ahat U = Q Y, the Arnoldi relation Ahat Q = Q H gives H = Y X^{-1};
//   * least squares min ||beta e_1 - H z|| after every panel (one-stage) or big panel
//     (two-stage); when the estimate falls to tol, or the restart length m is
//     reached, y += Q z and the cycle restarts from the true residual;
//   * convergence is declared on the true relative residual ||b - A x|| / ||b||.
#include "krylov.hpp"

namespace oracle {

std::vector<double> spmv(const Csr& A, const std::vector<double>& x) {
  std::vector<double> y((size_t)A.n, 0.0);
  for (int64_t i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int64_t k = A.rowptr[(size_t)i]; k < A.rowptr[(size_t)i + 1]; ++k)
      s += A.val[(size_t)k] * x[(size_t)A.col[(size_t)k]];
    y[(size_t)i] = s;
  }
  return y;
}

// [Ahat u, Ahat^2 u, ..., Ahat^s u] (Section 4, monomial basis)
Mat mpk(const Csr& A, const std::vector<double>& u, int s) {
  Mat V(A.n, s);
  std::vector<double> v = u;
  for (int i = 0; i < s; ++i) {
    v = spmv(A, v);
    for (int64_t r = 0; r < A.n; ++r) V(r, i) = v[(size_t)r];
  }
  return V;
}

static double norm2(const std::vector<double>& v) {
  double s = 0.0;
  for (double x : v) s += x * x;
  return std::sqrt(s);
}

// Ahat = A D^{-1} and D^{-1} for the right Jacobi preconditioner (or A and ones)
static Csr scaled(const Csr& A, bool jacobi, std::vector<double>& dinv) {
  Csr B = A;
  dinv.assign((size_t)A.n, 1.0);
  if (!jacobi) return B;
  for (int64_t i = 0; i < A.n; ++i) {
    double dg = 0.0;
    for (int64_t k = A.rowptr[(size_t)i]; k < A.rowptr[(size_t)i + 1]; ++k)
      if (A.col[(size_t)k] == i) dg += A.val[(size_t)k];
    if (dg == 0.0) throw std::runtime_error("Jacobi preconditioner needs a nonzero diagonal");
    dinv[(size_t)i] = 1.0 / dg;
  }
  for (size_t k = 0; k < B.val.size(); ++k) B.val[k] *= dinv[(size_t)B.col[k]];
  return B;
}

// min ||beta e_1 - H z|| for the (k + 1) x k Hessenberg H by Householder QR: z solves
// R z = Q^T g; the returned estimate is ||g - H z|| evaluated directly.
static std::vector<double> least_squares(const Mat& H, double beta, double& est) {
  const int64_t k = H.n;
  Mat R, Q;
  householder_qr(H, R, &Q);
  std::vector<double> z((size_t)k, 0.0);
  for (int64_t i = k - 1; i >= 0; --i) {
    double v = Q(0, i) * beta;
    for (int64_t l = i + 1; l < k; ++l) v -= R(i, l) * z[(size_t)l];
    z[(size_t)i] = v / R(i, i);
  }
  double ss = 0.0;
  for (int64_t i = 0; i < H.m; ++i) {
    double v = i == 0 ? beta : 0.0;
    for (int64_t l = 0; l < k; ++l) v -= H(i, l) * z[(size_t)l];
    ss += v * v;
  }
  est = std::sqrt(ss);
  return z;
}

GmresResult sstep_gmres(const Csr& A, const std::vector<double>& b, int s, int m, double tol, int scheme,
                        int s_hat, int intra, int pip, int d, int zeta, uint64_t seed, int max_restarts,
                        bool jacobi) {
  std::vector<double> dinv;
  const Csr Ah = scaled(A, jacobi, dinv);
  const int64_t n = A.n;
  if (m % s != 0) throw std::runtime_error("m must be a multiple of s");
  if (scheme == 1 && (s_hat < s || m % s_hat != 0 || s_hat % s != 0))
    throw std::runtime_error("need s | s_hat | m");
  const Sketch S(n, d, zeta, seed);
  const double bnorm = norm2(b);
  std::vector<double> y((size_t)n, 0.0);
  GmresResult res;
  int its = 0;
  for (int cycle = 0; cycle <= max_restarts; ++cycle) {
    std::vector<double> r = spmv(Ah, y);
    for (int64_t i = 0; i < n; ++i) r[(size_t)i] = b[(size_t)i] - r[(size_t)i];
    Mat rr(n, 1), q0, r00;
    for (int64_t i = 0; i < n; ++i) rr(i, 0) = r[(size_t)i];
    try {
      cholqr(rr, q0, r00, "v0");
    } catch (const Breakdown&) {  // r == 0
      res.converged = true;
      res.relres = 0.0;
      break;
    }
    const double beta = r00(0, 0), rel = beta / bnorm;
    res.history.push_back({its, rel});
    res.relres = rel;
    if (rel <= tol) {
      res.converged = true;
      break;
    }
    if (cycle == max_restarts) break;
    res.restarts = cycle;
    Mat Qb(n, m + 1), R(m + 1, m + 1), X(m, m), Y(m + 1, m);
    for (int64_t i = 0; i < n; ++i) Qb(i, 0) = q0(i, 0);
    R(0, 0) = beta;
    int ncols = 1;
    std::vector<double> z;
    try {
      while (ncols < m + 1) {
        const int P = ncols;
        std::vector<double> u((size_t)n);
        for (int64_t i = 0; i < n; ++i) u[(size_t)i] = Qb(i, P - 1);
        if (scheme == 0) {
          Mat Qj, Rtop, Rjj;
          bcgs2_block(cols(Qb, 0, P), mpk(Ah, u, s), intra, &S, Qj, Rtop, Rjj);
          for (int j = 0; j < s; ++j) {
            for (int64_t i = 0; i < n; ++i) Qb(i, P + j) = Qj(i, j);
            for (int i = 0; i < P; ++i) R(i, P + j) = Rtop(i, j);
            for (int i = 0; i < s; ++i) R(P + i, P + j) = Rjj(i, j);
          }
          X(P - 1, P - 1) = 1.0;
          for (int i = 1; i < s; ++i)
            for (int t = 0; t < P + i; ++t) X(t, P - 1 + i) = R(t, P + i - 1);
          for (int j = 0; j < s; ++j)
            for (int t = 0; t < P + s; ++t) Y(t, P - 1 + j) = R(t, P + j);
          ncols += s;
          its += s;
        } else {
          const Mat Qp = cols(Qb, 0, P);
          TwoStageBigPanel bp(Qp, pip ? nullptr : &S, s_hat, pip);
          std::vector<int> gens;
          for (int j = 0; j < s_hat / s; ++j) {
            if (j > 0) {
              for (int64_t i = 0; i < n; ++i) u[(size_t)i] = bp.Qbar(i, bp.Qbar.n - 1);
              gens.push_back(bp.cols - 1);
            } else {
              gens.push_back(-1);
            }
            bp.add_panel(mpk(Ah, u, s));
          }
          Mat QB, RQB, RBB, cq;
          bp.finish(QB, RQB, RBB, cq);
          for (int j = 0; j < s_hat; ++j) {
            for (int64_t i = 0; i < n; ++i) Qb(i, P + j) = QB(i, j);
            for (int i = 0; i < P; ++i) R(i, P + j) = RQB(i, j);
            for (int i = 0; i < s_hat; ++i) R(P + i, P + j) = RBB(i, j);
          }
          for (size_t j = 0; j < gens.size(); ++j) {
            const int c = P + (int)j * s, g = gens[j];
            if (g < 0) X(c - 1, c - 1) = 1.0;
            else
              for (int t = 0; t < P + g + 1; ++t) X(t, c - 1) = cq(t, g);
            for (int i = 1; i < s; ++i)
              for (int t = 0; t < c + i; ++t) X(t, c - 1 + i) = R(t, c + i - 1);
          }
          for (int j = 0; j < s_hat; ++j)
            for (int t = 0; t < P + s_hat; ++t) Y(t, P - 1 + j) = R(t, P + j);
          ncols += s_hat;
          its += s_hat;
        }
        const int k = ncols - 1;
        Mat Yk(ncols, k), Xk(k, k);
        for (int j = 0; j < k; ++j) {
          for (int t = 0; t < ncols; ++t) Yk(t, j) = Y(t, j);
          for (int t = 0; t < k; ++t) Xk(t, j) = X(t, j);
        }
        double est = 0.0;
        z = least_squares(solve_right_upper(Yk, Xk), beta, est);
        if (est / bnorm <= tol) break;
      }
    } catch (const Breakdown&) {
      res.breakdown = true;
      res.iterations = its;
      res.x.assign((size_t)n, 0.0);
      for (int64_t i = 0; i < n; ++i) res.x[(size_t)i] = dinv[(size_t)i] * y[(size_t)i];
      return res;
    }
    const int k = ncols - 1;
    for (int64_t i = 0; i < n; ++i) {
      double v = 0.0;
      for (int j = 0; j < k; ++j) v += Qb(i, j) * z[(size_t)j];
      y[(size_t)i] += v;
    }
  }
  res.iterations = its;
  res.x.assign((size_t)n, 0.0);
  for (int64_t i = 0; i < n; ++i) res.x[(size_t)i] = dinv[(size_t)i] * y[(size_t)i];
  return res;
}

// GMRES(m) with Householder-reflector Arnoldi (Walker, SISC 9, 1988), the most stable
// formulation: the brute-force reference for small n.
GmresResult householder_gmres(const Csr& A, const std::vector<double>& b, int m, double tol,
                              int max_restarts, bool jacobi) {
  std::vector<double> dinv;
  const Csr Ah = scaled(A, jacobi, dinv);
  const int64_t n = A.n;
  const double bnorm = norm2(b);
  std::vector<double> y((size_t)n, 0.0);
  GmresResult res;
  int its = 0;
  auto reflect = [&](const std::vector<double>& w, std::vector<double>& v) {  // v -= 2 w (w . v)
    double t = 0.0;
    for (int64_t i = 0; i < n; ++i) t += w[(size_t)i] * v[(size_t)i];
    for (int64_t i = 0; i < n; ++i) v[(size_t)i] -= 2.0 * w[(size_t)i] * t;
  };
  for (int cycle = 0; cycle <= max_restarts; ++cycle) {
    std::vector<double> r = spmv(Ah, y);
    for (int64_t i = 0; i < n; ++i) r[(size_t)i] = b[(size_t)i] - r[(size_t)i];
    const double rel = norm2(r) / bnorm;
    res.history.push_back({its, rel});
    res.relres = rel;
    if (rel <= tol) {
      res.converged = true;
      break;
    }
    if (cycle == max_restarts) break;
    res.restarts = cycle;
    std::vector<std::vector<double>> W;
    Mat H(m + 1, m);
    std::vector<double> zv = r, z;
    double g0 = 0.0;
    int kdone = 0;
    for (int j = 0; j <= m; ++j) {
      std::vector<double> w = zv;
      for (int i = 0; i < j; ++i) w[(size_t)i] = 0.0;
      double ss = 0.0;
      for (int64_t i = j; i < n; ++i) ss += w[(size_t)i] * w[(size_t)i];
      const double alpha = std::sqrt(ss);
      if (alpha == 0.0) break;
      w[(size_t)j] += (w[(size_t)j] >= 0.0 ? 1.0 : -1.0) * alpha;
      const double wn = norm2(w);
      for (double& x : w) x /= wn;
      W.push_back(w);
      std::vector<double> h = zv;
      reflect(w, h);
      if (j == 0) {
        g0 = h[0];
      } else {
        for (int i = 0; i <= j; ++i) H(i, j - 1) = h[(size_t)i];
        kdone = j;
        Mat Hj(j + 1, j);
        for (int c = 0; c < j; ++c)
          for (int i = 0; i <= j; ++i) Hj(i, c) = H(i, c);
        double est = 0.0;
        z = least_squares(Hj, g0, est);
        ++its;
        if (est / bnorm <= tol) break;
      }
      if (j == m) break;
      std::vector<double> q((size_t)n, 0.0);
      q[(size_t)j] = 1.0;
      for (int i = j; i >= 0; --i) reflect(W[(size_t)i], q);
      zv = spmv(Ah, q);
      for (int i = 0; i <= j; ++i) reflect(W[(size_t)i], zv);
    }
    for (int i = 0; i < kdone; ++i) {
      std::vector<double> q((size_t)n, 0.0);
      q[(size_t)i] = 1.0;
      for (int t = i; t >= 0; --t) reflect(W[(size_t)t], q);
      for (int64_t l = 0; l < n; ++l) y[(size_t)l] += z[(size_t)i] * q[(size_t)l];
    }
  }
  res.iterations = its;
  res.x.assign((size_t)n, 0.0);
  for (int64_t i = 0; i < n; ++i) res.x[(size_t)i] = dinv[(size_t)i] * y[(size_t)i];
  return res;
}

}  // namespace oracle

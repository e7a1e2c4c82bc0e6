// C interface of the C++ oracle (test infrastructure); see oracle_c.h.
#include "oracle_c.h"

#include <algorithm>

#include "krylov.hpp"

using namespace oracle;

static Mat load(int64_t m, int64_t n, const double* p) {
  Mat A(m, n);
  std::memcpy(A.a.data(), p, sizeof(double) * (size_t)(m * n));
  return A;
}
static void store(const Mat& A, double* p) { std::memcpy(p, A.a.data(), sizeof(double) * A.a.size()); }
static Csr csr(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val) {
  Csr A;
  A.n = n;
  A.rowptr.assign(rowptr, rowptr + n + 1);
  A.col.assign(col, col + rowptr[n]);
  A.val.assign(val, val + rowptr[n]);
  return A;
}
static void results(const GmresResult& r, double* x, int32_t* stats, double* relres, double* history,
                    int32_t hist_cap) {
  std::memcpy(x, r.x.data(), sizeof(double) * r.x.size());
  const int32_t h = (int32_t)std::min<size_t>(r.history.size(), (size_t)hist_cap);
  for (int32_t i = 0; i < h; ++i) {
    history[2 * i] = r.history[(size_t)i].first;
    history[2 * i + 1] = r.history[(size_t)i].second;
  }
  stats[0] = r.iterations;
  stats[1] = r.restarts;
  stats[2] = r.converged ? 1 : 0;
  stats[3] = r.breakdown ? 1 : 0;
  stats[4] = h;
  *relres = r.relres;
}

#define GUARD(body)          \
  try {                      \
    body;                    \
    return 0;                \
  } catch (...) {            \
    return -1;               \
  }

extern "C" {

uint64_t orc_splitmix64(uint64_t seed, uint64_t i) { return splitmix64_output(seed, i); }

int orc_sparse_sign_entries(int64_t row0, int64_t nrows, int32_t d, int32_t zeta, uint64_t seed,
                            int32_t* idx, int8_t* sgn) {
  return sparse_sign_entries(row0, nrows, d, zeta, seed, idx, sgn) ? 0 : -1;
}

int orc_sketch_apply(int64_t n, int32_t d, int32_t zeta, uint64_t seed, int32_t k, const double* W,
                     double* out) {
  GUARD(store(Sketch(n, d, zeta, seed).apply(load(n, k, W)), out))
}

double orc_gaussian_entry(uint64_t seed, uint64_t r, int32_t k, int32_t d) { return gaussian_entry(seed, r, k, d); }

int orc_cholesky_upper(int32_t k, const double* G, double* R) {
  Mat Rm;
  const int info = cholesky_upper(load(k, k, G), Rm);
  store(Rm, R);
  return info;
}

int orc_householder_qr(int64_t m, int32_t k, const double* A, double* R, double* Q) {
  GUARD(Mat Rm; Mat Qm; householder_qr(load(m, k, A), Rm, Q ? &Qm : nullptr); store(Rm, R);
        if (Q) store(Qm, Q))
}

int orc_solve_right_upper(int64_t m, int32_t k, const double* W, const double* R, double* X) {
  GUARD(store(solve_right_upper(load(m, k, W), load(k, k, R)), X))
}

int orc_gram(int64_t n, int32_t a, const double* X, int32_t b, const double* Y, double* C) {
  GUARD(store(gram(load(n, a, X), load(n, b, Y)), C))
}

double orc_orth_error(int64_t n, int32_t c, const double* Q) { return orth_error(load(n, c, Q)); }

double orc_backward_error(int64_t n, int32_t c, const double* V, const double* Q, const double* R) {
  return backward_error(load(n, c, V), load(n, c, Q), load(c, c, R));
}

int orc_block_orth(int32_t scheme, int64_t n, int32_t c, int32_t s, int32_t s_hat, int32_t intra,
                   int32_t pip, int32_t v0, int32_t d, int32_t zeta, uint64_t seed, const double* V,
                   double* Q, double* R, int32_t* info) {
  GUARD(const Mat Vm = load(n, c, V);
        const bool sketched = scheme == 0 ? intra == 0 : pip == 0;
        Sketch* S = sketched ? new Sketch(n, d, zeta, seed) : nullptr;
        OrthResult o;
        try {
          o = scheme == 0 ? block_orth_one_stage(Vm, s, S, intra, v0 != 0)
                          : block_orth_two_stage(Vm, s, s_hat, S, v0 != 0, pip);
        } catch (...) {
          delete S;
          throw;
        }
        delete S; store(o.Q, Q); store(o.R, R); info[0] = o.ok ? 1 : 0; info[1] = o.breakdown_block;
        info[2] = o.breakdown_column)
}

int orc_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
             double* y) {
  GUARD(const std::vector<double> yy = spmv(csr(n, rowptr, col, val), std::vector<double>(x, x + n));
        std::memcpy(y, yy.data(), sizeof(double) * (size_t)n))
}

int orc_sstep_gmres(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                    const double* b, int32_t s, int32_t m, double tol, int32_t scheme, int32_t s_hat,
                    int32_t intra, int32_t pip, int32_t d, int32_t zeta, uint64_t seed,
                    int32_t max_restarts, int32_t jacobi, double* x, int32_t* stats, double* relres,
                    double* history, int32_t hist_cap) {
  GUARD(const GmresResult r = sstep_gmres(csr(n, rowptr, col, val), std::vector<double>(b, b + n), s, m, tol,
                                          scheme, s_hat, intra, pip, d, zeta, seed, max_restarts, jacobi != 0);
        results(r, x, stats, relres, history, hist_cap))
}

int orc_householder_gmres(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                          const double* b, int32_t m, double tol, int32_t max_restarts, int32_t jacobi,
                          double* x, int32_t* stats, double* relres, double* history, int32_t hist_cap) {
  GUARD(const GmresResult r = householder_gmres(csr(n, rowptr, col, val), std::vector<double>(b, b + n), m, tol,
                                                max_restarts, jacobi != 0);
        results(r, x, stats, relres, history, hist_cap))
}

}  // extern "C"

// CSR SpMV, monomial matrix-powers kernel, s-step GMRES and Householder GMRES of the
// oracle (test infrastructure); see krylov.cpp.
#pragma once

#include <utility>

#include "orth.hpp"

namespace oracle {

struct Csr {
  int64_t n = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
};

std::vector<double> spmv(const Csr& A, const std::vector<double>& x);
Mat mpk(const Csr& A, const std::vector<double>& u, int s);

struct GmresResult {
  std::vector<double> x;
  bool converged = false;
  int iterations = 0, restarts = 0;
  double relres = INFINITY;
  std::vector<std::pair<int, double>> history;  // (iterations, true relative residual)
  bool breakdown = false;
};

// scheme 0: one-stage (intra 0 RandCholQR, 1 CholQR2); scheme 1: two-stage with big
// panels of s_hat (pip 0 RandBCGS2, 1 BCGS-PIP).  Jacobi right preconditioning when
// jacobi, monomial basis.
GmresResult sstep_gmres(const Csr& A, const std::vector<double>& b, int s, int m, double tol, int scheme,
                        int s_hat, int intra, int pip, int d, int zeta, uint64_t seed, int max_restarts,
                        bool jacobi);
GmresResult householder_gmres(const Csr& A, const std::vector<double>& b, int m, double tol,
                              int max_restarts, bool jacobi);

}  // namespace oracle

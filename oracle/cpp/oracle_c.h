/* C interface of the C++ oracle (TEST INFRASTRUCTURE ONLY: loaded by the tests through
 * oracle/cpp_oracle.py, never by the library).  Every matrix is column-major and
 * contiguous (leading dimension = its row count); the caller owns every array.
 * Functions return 0 on success and -1 when the computation threw (invalid shapes, a
 * sketch row without zeta distinct indices); a Cholesky breakdown is a result, not an
 * error, and is reported through the `info` outputs. */
#pragma once
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

uint64_t orc_splitmix64(uint64_t seed, uint64_t i);
int orc_sparse_sign_entries(int64_t row0, int64_t nrows, int32_t d, int32_t zeta, uint64_t seed,
                            int32_t* idx, int8_t* sgn);
/* out (d x k) = S W, S the n-column sparse-sign sketch, W n x k */
int orc_sketch_apply(int64_t n, int32_t d, int32_t zeta, uint64_t seed, int32_t k, const double* W,
                     double* out);
double orc_gaussian_entry(uint64_t seed, uint64_t r, int32_t k, int32_t d);
/* R (k x k) with G = R^T R; returns -1 or the breaking column */
int orc_cholesky_upper(int32_t k, const double* G, double* R);
/* A m x k -> R (k x k, non-negative diagonal) and, if Q is not null, Q (m x k) */
int orc_householder_qr(int64_t m, int32_t k, const double* A, double* R, double* Q);
int orc_solve_right_upper(int64_t m, int32_t k, const double* W, const double* R, double* X);
int orc_gram(int64_t n, int32_t a, const double* X, int32_t b, const double* Y, double* C);
double orc_orth_error(int64_t n, int32_t c, const double* Q);
double orc_backward_error(int64_t n, int32_t c, const double* V, const double* Q, const double* R);
/* scheme 0: one-stage (intra 0 RandCholQR, 1 CholQR2); 1: two-stage with big panels of
 * s_hat (pip 0 RandBCGS2, 1 BCGS-PIP).  Q (n x c), R (c x c); info = {ok, breakdown
 * block, breakdown column} */
int orc_block_orth(int32_t scheme, int64_t n, int32_t c, int32_t s, int32_t s_hat, int32_t intra,
                   int32_t pip, int32_t v0, int32_t d, int32_t zeta, uint64_t seed, const double* V,
                   double* Q, double* R, int32_t* info);
int orc_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
             double* y);
/* stats = {iterations, restarts, converged, breakdown, history pairs written}; history
 * holds (iteration, relative residual) pairs, at most hist_cap */
int orc_sstep_gmres(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                    const double* b, int32_t s, int32_t m, double tol, int32_t scheme, int32_t s_hat,
                    int32_t intra, int32_t pip, int32_t d, int32_t zeta, uint64_t seed,
                    int32_t max_restarts, int32_t jacobi, double* x, int32_t* stats, double* relres,
                    double* history, int32_t hist_cap);
int orc_householder_gmres(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                          const double* b, int32_t m, double tol, int32_t max_restarts, int32_t jacobi,
                          double* x, int32_t* stats, double* relres, double* history, int32_t hist_cap);

#ifdef __cplusplus
}
#endif

// s-step GMRES (Section 4, Figure 1) driver: right preconditioning, monomial
// matrix-powers kernel, one-stage or two-stage randomized block orthogonalization,
// Hessenberg H = Y X^{-1} from the R factors and a Givens least-squares solve on
// the host.
//
// With generators U (the vectors the operator is applied to) and outputs
// W = Ahat U, written in the orthonormal basis as U = Q X and W = Q Y, the Arnoldi
// relation Ahat Q = Q H gives H = Y X^{-1}.  X is upper triangular: the first
// generator of a panel is the last orthonormal column (one-stage) or the last
// preprocessed column qbar (two-stage, inside a big panel), the others are the raw
// MPK outputs, whose coordinates are columns of R.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "rbo_internal.cuh"

namespace rbo {

// min || beta e1 - H z || for the (k+1) x k Hessenberg H (column-major, ld ldh)
// by Givens rotations; returns the residual norm and z.
static double hessenberg_ls(const std::vector<double>& Hin, int ldh, int k, double beta,
                            std::vector<double>& z) {
  std::vector<double> H(Hin.begin(), Hin.begin() + (size_t)ldh * k);
  std::vector<double> g(k + 1, 0.0);
  g[0] = beta;
  for (int j = 0; j < k; ++j) {
    // H(j+1, j) is the only subdiagonal entry (earlier rotations applied below)
    double a = H[j + (size_t)j * ldh], b = H[(j + 1) + (size_t)j * ldh];
    double r = std::hypot(a, b);
    double c = r == 0.0 ? 1.0 : a / r, s = r == 0.0 ? 0.0 : b / r;
    for (int l = j; l < k; ++l) {
      double h1 = H[j + (size_t)l * ldh], h2 = H[(j + 1) + (size_t)l * ldh];
      H[j + (size_t)l * ldh] = c * h1 + s * h2;
      H[(j + 1) + (size_t)l * ldh] = -s * h1 + c * h2;
    }
    double g1 = g[j], g2 = g[j + 1];
    g[j] = c * g1 + s * g2;
    g[j + 1] = -s * g1 + c * g2;
  }
  z.assign(k, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    double v = g[i];
    for (int l = i + 1; l < k; ++l) v -= H[i + (size_t)l * ldh] * z[l];
    z[i] = v / H[i + (size_t)i * ldh];
  }
  return std::fabs(g[k]);
}

struct GmresWork {
  double* Qb;       // n x (m+1), ld ldq
  int64_t ldq;
  double* vals;     // scaled CSR values (Jacobi)
  double* dscale;   // 1 / diag(A)
  double* t1;       // temporaries (n)
  double* t2;
  double* zdev;     // m
  double* Rdev;     // (m+1) x (m+1)
  double* coords;   // (m+1) x s_hat
  double* bn;       // 1 (||b||^2)
  // SELL-32 copy of the MPK operator (short rows, no separate M): slot offsets, slice
  // widths, indices and values
  int64_t* sell_off;
  int32_t* sell_w;
  int32_t* sell_col;
  double* sell_val;
  int64_t sell_cap;
};

int sstep_gmres_impl(const rbo_csr* A, const double* Mval, const double* b, double* x, int s,
                     int s_hat, int m, double tol, int d, int zeta, uint64_t seed, int sk_type,
                     int d_inner, const rbo_opts* opts, rbo_info* info, cudaStream_t st,
                     int* launches_out) {
  const int64_t n = A->n;
  const bool two = s_hat > s;
  const int K = two ? s_hat : s;
  // 0: none, 1: Jacobi (scaled copy of the values), 2: M on A's pattern (Mval)
  const int precond = Mval ? 2 : (opts ? (opts->precond ? 1 : 0) : 1);
  const int max_restarts = (opts && opts->max_restarts > 0) ? opts->max_restarts : 1000;
  // first intra-block step of the one-stage scheme (the two-stage one is sketched)
  const int intra = opts ? opts->intra : RBO_INTRA_RANDCHOLQR;
  const int ld = m + 1;
  const int64_t ldq = (n + 1) & ~int64_t(1);  // even: 16-byte aligned columns

  const int pmax = m + 1, kmax = K;
  const int maxL = std::max(orth_max_L(pmax, kmax, std::max(d, d_inner)), 1);
  size_t bytes = reduction_bytes(maxL) + orth_ctx_bytes(pmax, kmax, d, n, zeta, sk_type, d_inner) +
                 (size_t)ldq * (m + 1) * 8 + (size_t)A->nnz * 8 + 2 * (size_t)n * 8 +
                 (size_t)(m + 1) * (m + 1) * 8 + (size_t)(m + 1) * K * 8 + (size_t)m * 8 + 16 * 1024;
  // the MPK operator in SELL-32 form when its rows are short (stencils): room for the
  // stored entries plus two padding slots per row on average
  const bool use_sell = precond != 2 && n > 0 && (double)A->nnz <= 12.0 * (double)n;
  const int64_t nsl = (n + 31) / 32;
  const int64_t sell_cap = use_sell ? A->nnz + 2 * n + 64 : 0;
  if (use_sell) bytes += (size_t)sell_cap * 12 + (size_t)(nsl + 1) * 8 + (size_t)nsl * 4 + 1024;
  Arena* ar = nullptr;
  int e = arena_prepare(&ar, bytes);
  if (e) return e;
  if ((e = arena_reserve_reduction(ar, maxL, st))) return e;
  GmresWork w;
  w.ldq = ldq;
  w.Qb = (double*)ar->take((size_t)ldq * (m + 1) * 8);
  w.vals = precond == 1 ? (double*)ar->take((size_t)std::max<int64_t>(A->nnz, 1) * 8) : nullptr;
  w.dscale = precond == 1 ? (double*)ar->take((size_t)n * 8) : nullptr;
  w.t1 = (double*)ar->take((size_t)n * 8);
  w.t2 = (double*)ar->take((size_t)n * 8);
  w.zdev = (double*)ar->take((size_t)m * 8 + 64);
  w.Rdev = (double*)ar->take((size_t)ld * ld * 8);
  w.coords = (double*)ar->take((size_t)ld * K * 8);
  w.bn = (double*)ar->take(64);
  w.sell_cap = sell_cap;
  w.sell_off = use_sell ? (int64_t*)ar->take((size_t)(nsl + 1) * 8) : nullptr;
  w.sell_w = use_sell ? (int32_t*)ar->take((size_t)nsl * 4) : nullptr;
  w.sell_col = use_sell ? (int32_t*)ar->take((size_t)sell_cap * 4) : nullptr;
  w.sell_val = use_sell ? (double*)ar->take((size_t)sell_cap * 8) : nullptr;
  if (use_sell && (!w.sell_off || !w.sell_w || !w.sell_col || !w.sell_val)) return RBO_ERR_NOMEM;
  if (!w.Qb || !w.t1 || !w.t2 || !w.zdev || !w.Rdev || !w.coords || !w.bn ||
      (precond == 1 && (!w.vals || !w.dscale)))
    return RBO_ERR_NOMEM;

  OrthCtx c;
  c.ar = ar;
  c.st = st;
  c.mixed = (opts && opts->precision == RBO_PREC_MIXED) ? 1 : 0;
  c.df64 = (opts && opts->precision == RBO_PREC_DF64) ? 1 : 0;
  c.ozaki = (opts && opts->precision == RBO_PREC_OZAKI) ? 1 : 0;
  c.pip = (two && opts && opts->preproc == RBO_PREPROC_PIP) ? 1 : 0;
  // the sketch is only needed by RandCholQR (one-stage) and RandBCGS2 (two-stage)
  const bool sketched = two ? !c.pip : intra == RBO_INTRA_RANDCHOLQR;
  c.d = sketched ? d : 0;
  c.zeta = zeta;
  c.seed = seed;
  c.sk_type = sk_type;
  c.d_inner = d_inner;
  if ((e = orth_ctx_alloc(c, pmax, kmax, n))) return e;

  CsrDev Araw{n, A->nnz, A->rowptr, A->col, A->val};
  CsrDev Ahat = Araw;
  CsrDev Mop{n, A->nnz, A->rowptr, A->col, Mval};
  if (precond == 1) {
    if ((e = jacobi_launch(Araw, w.dscale, ar->status, st))) return e;
    if ((e = scale_columns_launch(Araw, w.dscale, w.vals, st))) return e;
    Ahat.val = w.vals;
    c.launches += 2;
  }
  SellDev sell;
  if (use_sell) {
    if ((e = sell_build(Ahat, w.sell_cap, w.sell_off, w.sell_w, w.sell_col, w.sell_val, ar->status, st, &sell)))
      return e;
    if (sell.n > 0) c.launches += 2;
  }
  // out = A M u: one SpMV with the column-scaled values (Jacobi), two SpMVs (M given),
  // or one SpMV with A (no preconditioner)
  // out = A M u (+ the basis shift of `sh`, fused into the last SpMV)
  auto apply_op = [&](const double* u, double* out, const SpmvShift& sh) -> int {
    int r;
    if (precond == 2) {
      if ((r = spmv_launch(Mop, nullptr, u, w.t2, ar->status, st))) return r;
      if ((r = spmv_launch(Araw, nullptr, w.t2, out, ar->status, st, sh))) return r;
      c.launches += 2;
      return RBO_OK;
    }
    c.launches += 1;
    if (sell.n > 0) return spmv_sell_launch(sell, Ahat.nnz, u, out, st, sh);
    return spmv_launch(Ahat, nullptr, u, out, ar->status, st, sh);
  };
  // ||b||
  {
    RowPass r;
    r.n = n; r.Y = const_cast<double*>(b); r.ldy = ldq; r.b = 1; r.acc_y = 1;
    r.epi.op = EPI_STORE_ALL; r.epi.out = w.bn;
    if ((e = rowpass_launch(r, ar, st, &c.launches))) return e;
  }
  double bn2 = 0.0;
  if (cudaMemcpyAsync(&bn2, w.bn, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return RBO_ERR_CUDA;
  if ((e = finish_status(ar, st, info))) return e;
  const double bnorm = std::sqrt(bn2);
  if (bnorm == 0.0) {
    if (cudaMemsetAsync(x, 0, (size_t)n * 8, st) != cudaSuccess) return RBO_ERR_CUDA;
    if (info) { info->converged = 1; info->relres = 0.0; }
    *launches_out = c.launches;
    return cudaStreamSynchronize(st) == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
  }

  std::vector<double> Rh((size_t)ld * ld), X((size_t)m * m), Y((size_t)ld * m), H((size_t)ld * m);
  std::vector<double> coords((size_t)ld * K), z;
  int its = 0;
  bool converged = false;
  double relres = INFINITY, est_rel = INFINITY;
  int cycle = 0, fallbacks = 0;
  // Newton and Chebyshev bases: recurrence parameters from the first cycle's Ritz
  // values (monomial until then).  The generators U of a panel satisfy
  // A M U = W + U B with B bidiagonal (alpha on the diagonal, -beta above it), so the
  // Hessenberg matrix is (Y + X B) X^{-1}.
  const int basis = opts ? opts->basis : RBO_BASIS_MONOMIAL;
  const bool poly_basis = basis != RBO_BASIS_MONOMIAL;
  std::vector<double> sh_a(s, 0.0), sh_b(s, 0.0);
  bool shifted = false;
  // output i of a panel from generators g_i (and g_{i-1})
  auto gen_step = [&](const double* gi, const double* gprev, double* out, int i) -> int {
    SpmvShift sh;
    if (shifted) {
      sh.u = gi;
      sh.a = -sh_a[i];
      sh.uprev = gprev;
      sh.b = sh_b[i];
    }
    return apply_op(gi, out, sh);
  };
  // Y(:, c0 + i) += alpha_i X(:, c0 + i) - beta_i X(:, c0 + i - 1)
  auto shift_columns = [&](int c0) {
    if (!shifted) return;
    for (int i = 0; i < s; ++i)
      for (int r = 0; r < m; ++r) {
        double v = sh_a[i] * X[r + (size_t)(c0 + i) * m];
        if (sh_b[i] != 0.0) v -= sh_b[i] * X[r + (size_t)(c0 + i - 1) * m];
        Y[r + (size_t)(c0 + i) * ld] += v;
      }
  };
  // Mixed precision: a block that the float32 sketch could not precondition (loss of
  // orthogonality or a Cholesky breakdown) makes the restart cycle start over in
  // float64, which stays on for the rest of the solve; x is only updated at the end of
  // a cycle, so the cycle is simply redone.
  auto fallback = [&](int code) -> bool {
    if (!c.mixed || (code != RBO_ERR_LOST_ORTHOGONALITY && code != RBO_ERR_CHOL_BREAKDOWN))
      return false;
    if (cudaMemsetAsync(ar->status, 0, sizeof(DevStatus), st) != cudaSuccess) return false;
    c.mixed = 0;
    ++fallbacks;
    if (info) {
      info->breakdown_block = -1;
      info->breakdown_column = -1;
      info->breakdown_stage = 0;
    }
    return true;
  };
  for (cycle = 0; cycle <= max_restarts; ++cycle) {
    const int its0 = its;
    const int resid_len0 = info ? info->resid_len : 0, hist_len0 = info ? info->history_len : 0;
    // r = b - Ahat y into basis column 0, q0 = r / ||r||
    if ((e = residual_launch(Araw, b, x, w.Qb, ar->status, st))) return e;
    if (info && info->resid && info->resid_len < info->resid_cap && info->resid_ld >= n) {
      if ((e = note_cuda(cudaMemcpyAsync(info->resid + (int64_t)info->resid_len * info->resid_ld,
                                         w.Qb, (size_t)n * 8, cudaMemcpyDeviceToDevice, st))))
        return e;
      info->resid_len++;
    }
    c.launches += 1;
    if (cudaMemsetAsync(w.Rdev, 0, (size_t)ld * ld * 8, st) != cudaSuccess) return RBO_ERR_CUDA;
    if ((e = normalise_column(c, n, w.Qb, w.Rdev, ld, 0))) return e;
    double beta = 0.0;
    if (cudaMemcpyAsync(&beta, w.Rdev, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return RBO_ERR_CUDA;
    e = finish_status(ar, st, info);
    if (e == RBO_ERR_CHOL_BREAKDOWN && info && info->breakdown_stage == RBO_STAGE_V0) {
      // r == 0 exactly
      relres = 0.0;
      converged = true;
      break;
    }
    if (e) return e;
    relres = beta / bnorm;
    if (info && info->history && info->history_len < info->history_cap) {
      info->history[2 * info->history_len] = its;
      info->history[2 * info->history_len + 1] = relres;
      info->history_len++;
    }
    if (relres <= tol) {
      converged = true;
      break;
    }
    if (cycle == max_restarts) break;
    std::fill(X.begin(), X.end(), 0.0);
    std::fill(Y.begin(), Y.end(), 0.0);
    int ncols = 1;
    int blk = 0;
    bool redo = false;
    // Newton / Chebyshev basis: the cycle that provides the Ritz values runs standard
    // GMRES (panels of one column, one-stage), which does not depend on the
    // conditioning of a monomial panel; later cycles use panels of s shifted vectors
    const int sc = (poly_basis && !shifted) ? 1 : s;
    while (ncols < m + 1) {
      const int P = ncols;
      if (!two || sc != s) {
        double* W = w.Qb + (int64_t)P * ldq;
        const double* u = w.Qb + (int64_t)(P - 1) * ldq;
        for (int i = 0; i < sc; ++i)
          if ((e = gen_step(i == 0 ? u : W + (int64_t)(i - 1) * ldq,
                            i == 0 ? nullptr : (i == 1 ? u : W + (int64_t)(i - 2) * ldq),
                            W + (int64_t)i * ldq, i)))
            return e;
        if ((e = one_stage_block(c, n, w.Qb, ldq, P, W, ldq, sc, intra, w.Rdev, ld, P, blk)))
          return e;
        if (cudaMemcpy2DAsync(Rh.data() + (size_t)P * ld, (size_t)ld * 8, w.Rdev + (size_t)P * ld,
                              (size_t)ld * 8, (size_t)(P + sc) * 8, sc, cudaMemcpyDeviceToHost,
                              st) != cudaSuccess)
          return RBO_ERR_CUDA;
        if ((e = finish_status(ar, st, info))) {
          if (fallback(e)) {
            redo = true;
            break;
          }
          return e;
        }
        X[(P - 1) + (size_t)(P - 1) * m] = 1.0;
        for (int i = 1; i < sc; ++i)
          for (int r = 0; r < P + i; ++r) X[r + (size_t)(P - 1 + i) * m] = Rh[r + (size_t)(P + i - 1) * ld];
        for (int i = 0; i < sc; ++i)
          for (int r = 0; r < P + sc; ++r) Y[r + (size_t)(P - 1 + i) * ld] = Rh[r + (size_t)(P + i) * ld];
        shift_columns(P - 1);
        ncols += sc;
        its += sc;
      } else {
        BigPanel bp;
        bp.n = n; bp.Q = w.Qb; bp.ldq = ldq; bp.P = P;
        bp.VB = w.Qb + (int64_t)P * ldq; bp.ldv = ldq; bp.K = K; bp.blk = blk;
        std::vector<int> gens;
        for (int j = 0; j < K / s; ++j) {
          const double* u;
          if (j == 0) {
            u = w.Qb + (int64_t)(P - 1) * ldq;
            gens.push_back(-1);
          } else {
            u = bp.VB + (int64_t)(bp.cols - 1) * ldq;
            gens.push_back(bp.cols - 1);
          }
          double* W = bp.VB + (int64_t)bp.cols * ldq;
          for (int i = 0; i < s; ++i)
            if ((e = gen_step(i == 0 ? u : W + (int64_t)(i - 1) * ldq,
                              i == 0 ? nullptr : (i == 1 ? u : W + (int64_t)(i - 2) * ldq),
                              W + (int64_t)i * ldq, i)))
              return e;
          if ((e = bigpanel_add(c, bp, s))) return e;
        }
        if ((e = bigpanel_finish(c, bp, w.Rdev, ld, P, w.coords, ld))) return e;
        if (cudaMemcpy2DAsync(Rh.data() + (size_t)P * ld, (size_t)ld * 8, w.Rdev + (size_t)P * ld,
                              (size_t)ld * 8, (size_t)(P + K) * 8, K, cudaMemcpyDeviceToHost,
                              st) != cudaSuccess)
          return RBO_ERR_CUDA;
        if (cudaMemcpy2DAsync(coords.data(), (size_t)ld * 8, w.coords, (size_t)ld * 8,
                              (size_t)(P + K) * 8, K, cudaMemcpyDeviceToHost, st) != cudaSuccess)
          return RBO_ERR_CUDA;
        if ((e = finish_status(ar, st, info))) {
          if (fallback(e)) {
            redo = true;
            break;
          }
          return e;
        }
        for (int j = 0; j < (int)gens.size(); ++j) {
          const int cc = P + j * s;  // first new column of panel j
          if (gens[j] < 0) {
            X[(cc - 1) + (size_t)(cc - 1) * m] = 1.0;
          } else {
            const int g = gens[j];
            for (int r = 0; r <= P + g; ++r) X[r + (size_t)(cc - 1) * m] = coords[r + (size_t)g * ld];
          }
          for (int i = 1; i < s; ++i)
            for (int r = 0; r < cc + i; ++r)
              X[r + (size_t)(cc - 1 + i) * m] = Rh[r + (size_t)(cc + i - 1) * ld];
        }
        for (int i = 0; i < K; ++i)
          for (int r = 0; r < P + K; ++r) Y[r + (size_t)(P - 1 + i) * ld] = Rh[r + (size_t)(P + i) * ld];
        for (int j = 0; j < (int)gens.size(); ++j) shift_columns(P - 1 + j * s);
        ncols += K;
        its += K;
      }
      ++blk;
      // H = Y X^{-1} on the first k = ncols-1 columns
      const int k = ncols - 1;
      for (int col = 0; col < k; ++col) {
        for (int r = 0; r < ncols; ++r) {
          double v = Y[r + (size_t)col * ld];
          for (int l = 0; l < col; ++l) v -= H[r + (size_t)l * ld] * X[l + (size_t)col * m];
          H[r + (size_t)col * ld] = v / X[col + (size_t)col * m];
        }
      }
      double est = hessenberg_ls(H, ld, k, beta, z);
      est_rel = est / bnorm;
      if (est_rel <= tol) break;
    }
    if (redo) {
      its = its0;
      if (info) {
        info->resid_len = resid_len0;
        info->history_len = hist_len0;
      }
      --cycle;
      continue;
    }
    // y += Q z
    const int k = ncols - 1;
    if (cudaMemcpyAsync(w.zdev, z.data(), (size_t)k * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return RBO_ERR_CUDA;
    // x += M (Q z)
    if ((e = gemv_update_launch(n, k, w.Qb, ldq, w.zdev, w.t1, 0, st))) return e;
    if (precond == 2) {
      if ((e = spmv_launch(Mop, nullptr, w.t1, w.t2, ar->status, st))) return e;
      if ((e = axpy_scaled_launch(n, nullptr, w.t2, x, st))) return e;
      c.launches += 3;
    } else {
      if ((e = axpy_scaled_launch(n, w.dscale, w.t1, x, st))) return e;
      c.launches += 2;
    }
    if (poly_basis && !shifted && k >= 1) {
      // Ritz values of the first cycle (kept monomial when the QR iteration fails)
      const int r = basis == RBO_BASIS_CHEBYSHEV
                        ? chebyshev_shifts(H.data(), ld, k, s, sh_a.data(), sh_b.data())
                        : newton_shifts(H.data(), ld, k, s, sh_a.data(), sh_b.data());
      if (r == RBO_OK) shifted = true;
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return RBO_ERR_CUDA;
  if (info) {
    info->iterations = its;
    info->restarts = cycle;
    info->converged = converged ? 1 : 0;
    info->relres = relres;
    info->est_relres = est_rel;
    info->fallbacks = fallbacks;
  }
  *launches_out = c.launches;
  return converged ? RBO_OK : RBO_ERR_NOT_CONVERGED;
}

}  // namespace rbo


static int sstep_gmres_entry(const rbo_csr* A, const double* Mval, const double* b, double* x,
                             int32_t s, int32_t s_hat, int32_t m, double tol, rbo_sketch sk,
                             const rbo_opts* opts, rbo_info* info, void* stream) {
  using namespace rbo;
  auto t0 = std::chrono::steady_clock::now();
  if (info) {
    double* h = info->history;
    int32_t cap = info->history_cap;
    double* rs = info->resid;
    int64_t rld = info->resid_ld;
    int32_t rcap = info->resid_cap;
    memset(info, 0, sizeof(*info));
    info->history = h;
    info->history_cap = cap;
    info->resid = rs;
    info->resid_ld = rld;
    info->resid_cap = rcap;
    info->breakdown_block = -1;
    info->breakdown_column = -1;
  }
  int code = RBO_OK;
  int launches = 0;
  if (!A || A->n < 1 || !A->rowptr || !A->col || !A->val || A->nnz < 0 || A->nnz >= (1LL << 31) ||
      !b || !x || s < 1 || m < s || m % s != 0 || m > 128 || !(tol > 0.0))
    code = RBO_ERR_ARG;
  if (s_hat == 0) s_hat = s;
  if (code == RBO_OK && (s_hat < s || s_hat % s != 0 || m % s_hat != 0 || s_hat > 64))
    code = RBO_ERR_ARG;
  if (code == RBO_OK && A->n < m + 1) code = RBO_ERR_ARG;
  const bool pip = s_hat > s && opts && opts->preproc == RBO_PREPROC_PIP;
  if (code == RBO_OK && opts && opts->preproc != RBO_PREPROC_RAND && opts->preproc != RBO_PREPROC_PIP)
    code = RBO_ERR_ARG;
  if (code == RBO_OK && !pip &&
      (sk ? !sketch_fits(sk, s) : (int64_t)4 * (m + 1) * s > MAX_SKETCH_DK))
    code = RBO_ERR_ARG;
  if (code == RBO_OK && !pip && (sk ? sk->d : 4 * (m + 1)) < s_hat) code = RBO_ERR_ARG;
  if (code == RBO_OK && opts && opts->precision != RBO_PREC_FP64 &&
      opts->precision != RBO_PREC_MIXED && opts->precision != RBO_PREC_DF64 &&
      opts->precision != RBO_PREC_OZAKI)
    code = RBO_ERR_ARG;
  if (code == RBO_OK && opts && opts->basis != RBO_BASIS_MONOMIAL && opts->basis != RBO_BASIS_NEWTON &&
      opts->basis != RBO_BASIS_CHEBYSHEV)
    code = RBO_ERR_ARG;
  if (code == RBO_OK && opts && opts->intra != RBO_INTRA_RANDCHOLQR &&
      (opts->intra != RBO_INTRA_CHOLQR2 || s_hat > s))
    code = RBO_ERR_ARG;
  int d = 4 * (m + 1), zeta = 8, sk_type = RBO_SKETCH_SPARSE_SIGN, d_inner = 0;
  uint64_t seed = 42;
  if (sk) {
    if (sk->n_max < A->n) code = RBO_ERR_ARG;
    d = sk->d;
    zeta = sk->zeta;
    seed = sk->seed;
    sk_type = sk->type;
    d_inner = sk->d_inner;
  }
  if (code == RBO_OK) {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) code = RBO_ERR_NO_DEVICE;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) code = RBO_ERR_NO_DEVICE;
  }
  if (code == RBO_OK)
    code = sstep_gmres_impl(A, Mval, b, x, s, s_hat, m, tol, d, zeta, seed, sk_type, d_inner, opts,
                            info, (cudaStream_t)stream, &launches);
  if (info) {
    info->status = code;
    info->kernel_launches = launches;
    info->time_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return code;
}

extern "C" int rbo_sstep_gmres(const rbo_csr* A, const double* b, double* x, int32_t s,
                               int32_t s_hat, int32_t m, double tol, rbo_sketch sk,
                               const rbo_opts* opts, rbo_info* info, void* stream) {
  return sstep_gmres_entry(A, nullptr, b, x, s, s_hat, m, tol, sk, opts, info, stream);
}

extern "C" int rbo_sstep_gmres_precond(const rbo_csr* A, const double* Mval, const double* b,
                                       double* x, int32_t s, int32_t s_hat, int32_t m, double tol,
                                       rbo_sketch sk, const rbo_opts* opts, rbo_info* info,
                                       void* stream) {
  if (!Mval) return RBO_ERR_ARG;
  return sstep_gmres_entry(A, Mval, b, x, s, s_hat, m, tol, sk, opts, info, stream);
}

// The C ABI (include/rbo.h): argument checking, the per-device workspace arena and
// the block-orthogonalization entry points.
#include <chrono>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "rbo_internal.cuh"

namespace rbo {

constexpr size_t ARENA_HEADER = 1024;   // status (64 B) + tickets
constexpr int MAX_DEVICES = 64;
static Arena g_arena[MAX_DEVICES];
static std::mutex g_arena_mu;

size_t reduction_bytes(int max_L) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  const size_t gmax = (size_t)8 * sms;  // <= 8 resident CTAs of 256 threads per SM
  const size_t ng = (gmax + 15) / 16;
  return (gmax + ng) * (size_t)max_L * 8 + 256;
}

int arena_prepare(Arena** out, size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RBO_ERR_NO_DEVICE;
  if (dev < 0 || dev >= MAX_DEVICES) return RBO_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_arena_mu);
  Arena& a = g_arena[dev];
  const size_t need = bytes + ARENA_HEADER + 4096;
  if (a.base == nullptr || a.cap < need) {
    if (a.base) {
      cudaDeviceSynchronize();
      cudaFree(a.base);
      a.base = nullptr;
      a.cap = 0;
    }
    size_t cap = need + need / 4;
    if (cudaMalloc(&a.base, cap) != cudaSuccess) {
      cudaGetLastError();
      a.base = nullptr;
      return RBO_ERR_NOMEM;
    }
    a.cap = cap;
    a.device = dev;
  }
  if (a.status_host == nullptr) {
    if (cudaMallocHost(&a.status_host, sizeof(DevStatus)) != cudaSuccess) {
      cudaGetLastError();
      return RBO_ERR_NOMEM;
    }
  }
  a.status = reinterpret_cast<DevStatus*>(a.base);
  a.tickets = reinterpret_cast<unsigned*>(a.base + 64);
  a.n_tickets = (int)((ARENA_HEADER - 64) / 4);
  a.reset();
  a.used = ARENA_HEADER;
  *out = &a;
  return RBO_OK;
}

int arena_reserve_reduction(Arena* ar, int max_L, cudaStream_t st) {
  const size_t rb = reduction_bytes(max_L);
  ar->red = (double*)ar->take(rb);
  if (!ar->red) return RBO_ERR_NOMEM;
  ar->red_bytes = rb;
  // zero the status word and every ticket of this call
  return note_cuda(cudaMemsetAsync(ar->base, 0, ARENA_HEADER, st));
}

int arena_release_current() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RBO_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_arena_mu);
  Arena& a = g_arena[dev];
  if (a.base) {
    cudaDeviceSynchronize();
    cudaFree(a.base);
  }
  if (a.status_host) cudaFreeHost(a.status_host);
  a = Arena();
  return RBO_OK;
}

static thread_local char g_last_error[256] = "";

int note_cuda(cudaError_t e) {
  if (e == cudaSuccess) return RBO_OK;
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return RBO_ERR_CUDA;
}

int finish_status(Arena* ar, cudaStream_t st, rbo_info* info) {
  int e = note_cuda(
      cudaMemcpyAsync(ar->status_host, ar->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  if (e) return e;
  if ((e = note_cuda(cudaStreamSynchronize(st)))) return e;
  if (prof_on()) prof_drain();
  const DevStatus& s = *ar->status_host;
  if (info) {
    info->breakdown_block = -1;
    info->breakdown_column = -1;
    info->breakdown_stage = 0;
    if (s.code == RBO_ERR_CHOL_BREAKDOWN || s.code == RBO_ERR_LOST_ORTHOGONALITY) {
      info->breakdown_block = s.block;
      info->breakdown_column = s.column;
      info->breakdown_stage = s.stage;
    }
  }
  return s.code;
}

// ---- sketch handles ----------------------------------------------------------------------
}  // namespace rbo


using namespace rbo;

static void info_clear(rbo_info* info) {
  if (!info) return;
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

static int info_done(rbo_info* info, int code, int launches,
                     std::chrono::steady_clock::time_point t0) {
  if (info) {
    info->status = code;
    info->kernel_launches = launches;
    info->time_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return code;
}

static int check_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RBO_ERR_NO_DEVICE;
  }
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return RBO_ERR_NO_DEVICE;
  return RBO_OK;
}

extern "C" {

const char* rbo_version(void) { return "rbo 0.1 (sm_103a)"; }

const char* rbo_last_error(void) { return rbo::g_last_error; }

const char* rbo_status_string(int s) {
  switch (s) {
    case RBO_OK: return "ok";
    case RBO_ERR_ARG: return "invalid argument";
    case RBO_ERR_CUDA: return "CUDA error";
    case RBO_ERR_CHOL_BREAKDOWN: return "Cholesky breakdown (non-positive pivot)";
    case RBO_ERR_NOT_CONVERGED: return "not converged";
    case RBO_ERR_TIMEOUT: return "device wait timed out";
    case RBO_ERR_SKETCH: return "sketch column without zeta distinct rows";
    case RBO_ERR_NOMEM: return "workspace allocation failed";
    case RBO_ERR_NO_DEVICE: return "no sm_103 CUDA device";
    case RBO_ERR_LOST_ORTHOGONALITY: return "loss of orthogonality in a block (first intra step failed)";
    default: return "unknown status";
  }
}

int rbo_release_workspace(void) { return arena_release_current(); }

int rbo_sketch_create(int64_t n_max, int32_t d, int32_t zeta, uint64_t seed, rbo_sketch* out) {
  if (!out || n_max < 0 || d < 1 || d > 4096 || zeta < 1 || zeta > 16 || zeta > d)
    return RBO_ERR_ARG;
  rbo_sketch s = new (std::nothrow) rbo_sketch_s;
  if (!s) return RBO_ERR_NOMEM;
  s->n_max = n_max;
  s->d = d;
  s->zeta = zeta;
  s->seed = seed;
  *out = s;
  return RBO_OK;
}

int rbo_sketch_create_ex(int64_t n_max, int32_t d, int32_t type, int32_t zeta, int32_t d_inner,
                         uint64_t seed, rbo_sketch* out) {
  if (!out || n_max < 0 || d < 1) return RBO_ERR_ARG;
  if (type == RBO_SKETCH_SPARSE_SIGN) {
    if (d > 4096 || zeta < 1 || zeta > 16 || zeta > d) return RBO_ERR_ARG;
    d_inner = 0;
  } else if (type == RBO_SKETCH_GAUSSIAN) {
    if (d > 256) return RBO_ERR_ARG;
    zeta = 0;
    d_inner = 0;
  } else if (type == RBO_SKETCH_COUNT_GAUSS) {
    if (d > 4096 || d_inner < 1 || d_inner > 4096) return RBO_ERR_ARG;
    zeta = 1;
  } else {
    return RBO_ERR_ARG;
  }
  rbo_sketch s = new (std::nothrow) rbo_sketch_s;
  if (!s) return RBO_ERR_NOMEM;
  s->n_max = n_max;
  s->d = d;
  s->zeta = zeta;
  s->seed = seed;
  s->type = type;
  s->d_inner = d_inner;
  *out = s;
  return RBO_OK;
}

int rbo_sketch_destroy(rbo_sketch sk) {
  delete sk;
  return RBO_OK;
}

int rbo_sketch_entries(rbo_sketch sk, int64_t row0, int64_t nrows, int32_t* idx, int8_t* sign,
                       void* stream) {
  if (!sk || row0 < 0 || nrows < 0 || (nrows > 0 && (!idx || !sign))) return RBO_ERR_ARG;
  if (sk->type == RBO_SKETCH_GAUSSIAN) return RBO_ERR_ARG;
  const int sd = sk->type == RBO_SKETCH_COUNT_GAUSS ? sk->d_inner : sk->d;
  int e = check_device();
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  Arena* ar = nullptr;
  if ((e = arena_prepare(&ar, 0))) return e;
  if (cudaMemsetAsync(ar->base, 0, ARENA_HEADER, st) != cudaSuccess) return RBO_ERR_CUDA;
  if ((e = sketch_entries_launch(row0, nrows, sd, sk->zeta, sk->seed, idx, sign, ar->status, st)))
    return e;
  return finish_status(ar, st, nullptr);
}

int rbo_sketch_apply(rbo_sketch sk, int64_t n, int32_t k, const double* W, int64_t ldw, double* out,
                     int32_t precision, void* stream) {
  if (!sk || n < 1 || n > sk->n_max || k < 1 || k > 64 || !W || ldw < n || !out) return RBO_ERR_ARG;
  if (!sketch_fits(sk, k)) return RBO_ERR_ARG;
  int e = check_device();
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  Arena* ar = nullptr;
  const int dmax = std::max(sk->d, sk->d_inner);
  const int L = orth_max_L(0, k, dmax);
  const size_t bytes = reduction_bytes(L) + (size_t)sk->d * k * 8 +
                       orth_ctx_bytes(0, k, sk->d, n, sk->zeta, sk->type, sk->d_inner) + 2048;
  if ((e = arena_prepare(&ar, bytes))) return e;
  if ((e = arena_reserve_reduction(ar, L, st))) return e;
  double* dout = (double*)ar->take((size_t)sk->d * k * 8);
  if (!dout) return RBO_ERR_NOMEM;
  OrthCtx c;
  c.ar = ar;
  c.st = st;
  c.d = sk->d; c.zeta = sk->zeta; c.seed = sk->seed; c.sk_type = sk->type; c.d_inner = sk->d_inner;
  if ((e = orth_ctx_alloc(c, 0, k, n))) return e;
  RowPass r;
  r.n = n; r.Y = const_cast<double*>(W); r.ldy = ldw; r.b = k;
  set_sketch(r, c);
  r.mixed = precision == RBO_PREC_MIXED ? 1 : 0;
  r.epi.op = EPI_SKETCH_OUT; r.epi.out_sk = dout;
  int launches = 0;
  if ((e = rowpass_launch(r, ar, st, &launches))) return e;
  if (cudaMemcpyAsync(out, dout, (size_t)sk->d * k * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return RBO_ERR_CUDA;
  return finish_status(ar, st, nullptr);
}

int rbo_gram(int64_t n, int32_t a, const double* X, int64_t ldx, int32_t b, const double* Y,
             int64_t ldy, double* C, void* stream) {
  return rbo_gram_ex(n, a, X, ldx, b, Y, ldy, C, RBO_PREC_FP64, stream);
}

int rbo_gram_ex(int64_t n, int32_t a, const double* X, int64_t ldx, int32_t b, const double* Y,
                int64_t ldy, double* C, int32_t precision, void* stream) {
  if (n < 1 || a < 1 || a > 128 || b < 1 || b > 64 || !X || !Y || !C || ldx < n || ldy < n ||
      a * b > 8192)
    return RBO_ERR_ARG;
  if (precision != RBO_PREC_FP64 && precision != RBO_PREC_OZAKI) return RBO_ERR_ARG;
  if (precision == RBO_PREC_OZAKI && (a > 64 || b > 8)) return RBO_ERR_ARG;
  int e = check_device();
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  Arena* ar = nullptr;
  const int L = a * b;
  if ((e = arena_prepare(&ar, reduction_bytes(L) + (size_t)L * 8 + 1024))) return e;
  if ((e = arena_reserve_reduction(ar, L, st))) return e;
  double* dout = (double*)ar->take((size_t)L * 8);
  RowPass r;
  r.n = n; r.X = X; r.ldx = ldx; r.a = a; r.Y = const_cast<double*>(Y); r.ldy = ldy; r.b = b;
  r.acc_x = 1;
  r.ozaki = precision == RBO_PREC_OZAKI ? 2 : 0;  // the caller asked for this kernel
  r.epi.op = EPI_STORE; r.epi.out = dout; r.epi.out_ld = a;
  int launches = 0;
  if ((e = rowpass_launch(r, ar, st, &launches))) return e;
  if (cudaMemcpyAsync(C, dout, (size_t)L * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return RBO_ERR_CUDA;
  return finish_status(ar, st, nullptr);
}


static int orth_common_checks(int64_t n, int32_t ncols, int32_t s, double* V, int64_t ldv, double* R,
                              int64_t ldr, const rbo_opts* opts) {
  const int v0 = (opts && opts->v0) ? 1 : 0;
  if (n < 1 || ncols < 1 || ncols > 129 || s < 1 || s > 64 || !V || ldv < n || !R || ldr < ncols)
    return RBO_ERR_ARG;
  if (n < ncols) return RBO_ERR_ARG;
  if ((ncols - v0) % s != 0) return RBO_ERR_ARG;
  if (opts && (opts->precision != RBO_PREC_FP64 && opts->precision != RBO_PREC_MIXED &&
               opts->precision != RBO_PREC_DF64 && opts->precision != RBO_PREC_OZAKI))
    return RBO_ERR_ARG;
  return RBO_OK;
}

static int copy_R_out(double* Rdev, int ncols, double* R, int64_t ldr, cudaStream_t st) {
  if (ldr == ncols)
    return cudaMemcpyAsync(R, Rdev, (size_t)ncols * ncols * 8, cudaMemcpyDeviceToHost, st) ==
                   cudaSuccess
               ? RBO_OK
               : RBO_ERR_CUDA;
  return cudaMemcpy2DAsync(R, (size_t)ldr * 8, Rdev, (size_t)ncols * 8, (size_t)ncols * 8, ncols,
                           cudaMemcpyDeviceToHost, st) == cudaSuccess
             ? RBO_OK
             : RBO_ERR_CUDA;
}

static int block_orth_impl(rbo_sketch sk, int64_t n, int32_t ncols, int32_t s, int32_t s_hat,
                           double* V, int64_t ldv, double* R, int64_t ldr, const rbo_opts* opts,
                           rbo_info* info, void* stream, int scheme /*0 one, 1 two*/, int intra) {
  auto t0 = std::chrono::steady_clock::now();
  info_clear(info);
  int e = orth_common_checks(n, ncols, s, V, ldv, R, ldr, opts);
  if (e) return info_done(info, e, 0, t0);
  const int preproc = (scheme == 1 && opts) ? opts->preproc : RBO_PREPROC_RAND;
  if (preproc != RBO_PREPROC_RAND && preproc != RBO_PREPROC_PIP) return info_done(info, RBO_ERR_ARG, 0, t0);
  const bool rand = scheme == 1 ? preproc == RBO_PREPROC_RAND : intra == RBO_INTRA_RANDCHOLQR;
  if (rand && (!sk || n > sk->n_max)) return info_done(info, RBO_ERR_ARG, 0, t0);
  if (rand && !sketch_fits(sk, s)) return info_done(info, RBO_ERR_ARG, 0, t0);
  if (rand && sk->d < (scheme == 1 ? s_hat : s)) return info_done(info, RBO_ERR_ARG, 0, t0);
  const int v0 = (opts && opts->v0) ? 1 : 0;
  if (scheme == 1) {
    if (s_hat < s || s_hat % s != 0 || (ncols - v0) % s_hat != 0 || s_hat > 64)
      return info_done(info, RBO_ERR_ARG, 0, t0);
  }
  if ((e = check_device())) return info_done(info, e, 0, t0);
  cudaStream_t st = (cudaStream_t)stream;
  const int d = rand ? sk->d : 0;
  const int kmax = scheme == 1 ? s_hat : s;
  const int pmax = ncols;
  const int maxL = orth_max_L(pmax, kmax, rand ? std::max(sk->d, sk->d_inner) : 0);
  Arena* ar = nullptr;
  const bool mixed = opts && opts->precision == RBO_PREC_MIXED;
  size_t bytes = reduction_bytes(maxL) +
                 orth_ctx_bytes(pmax, kmax, d, n, rand ? sk->zeta : 0, rand ? sk->type : 0,
                                rand ? sk->d_inner : 0) +
                 (size_t)ncols * ncols * 8 + 4096;
  if (mixed) bytes += (size_t)n * kmax * 8 + 256;  // copy of the block in flight
  if ((e = arena_prepare(&ar, bytes))) return info_done(info, e, 0, t0);
  if ((e = arena_reserve_reduction(ar, maxL, st))) return info_done(info, e, 0, t0);
  double* Rdev = (double*)ar->take((size_t)ncols * ncols * 8);
  if (!Rdev) return info_done(info, RBO_ERR_NOMEM, 0, t0);
  if (cudaMemsetAsync(Rdev, 0, (size_t)ncols * ncols * 8, st) != cudaSuccess)
    return info_done(info, RBO_ERR_CUDA, 0, t0);
  OrthCtx c;
  c.ar = ar;
  c.st = st;
  c.mixed = (opts && opts->precision == RBO_PREC_MIXED) ? 1 : 0;
  c.df64 = (opts && opts->precision == RBO_PREC_DF64) ? 1 : 0;
  c.ozaki = (opts && opts->precision == RBO_PREC_OZAKI) ? 1 : 0;
  c.pip = preproc == RBO_PREPROC_PIP ? 1 : 0;
  if (rand) {
    c.d = sk->d;
    c.zeta = sk->zeta;
    c.seed = sk->seed;
    c.sk_type = sk->type;
    c.d_inner = sk->d_inner;
  }
  if ((e = orth_ctx_alloc(c, pmax, kmax, n))) return info_done(info, e, 0, t0);
  // Mixed precision: a block (two-stage: a big panel) that the float32 steps could not
  // precondition -- its final CholQR lost orthogonality or a Cholesky pivot broke down --
  // is redone in float64 from a copy of its columns taken before it started, and float64
  // stays on for the rest of the call (as in s-step GMRES).  In this mode every block
  // ends with a status check (one synchronisation of the stream).
  double* save = nullptr;
  if (mixed && !(save = (double*)ar->take((size_t)n * kmax * 8))) return info_done(info, RBO_ERR_NOMEM, 0, t0);
  int fallbacks = 0;
  auto guarded = [&](int p0, int width, auto&& body) -> int {
    double* Vb = V + (int64_t)p0 * ldv;
    const bool guard = c.mixed != 0;
    if (guard && cudaMemcpy2DAsync(save, (size_t)n * 8, Vb, (size_t)ldv * 8, (size_t)n * 8, width,
                                   cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return note_cuda(cudaGetLastError());
    int e2 = body();
    if (e2 || !guard) return e2;
    if ((e2 = note_cuda(cudaMemcpyAsync(ar->status_host, ar->status, sizeof(DevStatus),
                                        cudaMemcpyDeviceToHost, st))))
      return e2;
    if ((e2 = note_cuda(cudaStreamSynchronize(st)))) return e2;
    const int code = ar->status_host->code;
    if (code != RBO_ERR_LOST_ORTHOGONALITY && code != RBO_ERR_CHOL_BREAKDOWN) return RBO_OK;
    if ((e2 = note_cuda(cudaMemsetAsync(ar->status, 0, sizeof(DevStatus), st)))) return e2;
    if ((e2 = note_cuda(cudaMemcpy2DAsync(Vb, (size_t)ldv * 8, save, (size_t)n * 8, (size_t)n * 8, width,
                                          cudaMemcpyDeviceToDevice, st))))
      return e2;
    c.mixed = 0;
    ++fallbacks;
    return body();
  };
  int p = 0;
  if (v0) {
    if ((e = normalise_column(c, n, V, Rdev, ncols, 0))) return info_done(info, e, c.launches, t0);
    p = 1;
  }
  if (scheme == 0) {
    int blk = 0;
    for (; p < ncols; p += s, ++blk) {
      e = guarded(p, s, [&]() {
        return one_stage_block(c, n, V, ldv, p, V + (int64_t)p * ldv, ldv, s, intra, Rdev, ncols, p, blk);
      });
      if (info) info->fallbacks = fallbacks;
      if (e) return info_done(info, e, c.launches, t0);
    }
  } else {
    int blk = 0;
    for (; p < ncols; p += s_hat, ++blk) {
      e = guarded(p, s_hat, [&]() {
        BigPanel bp;
        bp.n = n; bp.Q = V; bp.ldq = ldv; bp.P = p;
        bp.VB = V + (int64_t)p * ldv; bp.ldv = ldv; bp.K = s_hat; bp.blk = blk;
        int e3 = RBO_OK;
        for (int j = 0; j < s_hat / s && !e3; ++j) e3 = bigpanel_add(c, bp, s);
        return e3 ? e3 : bigpanel_finish(c, bp, Rdev, ncols, p, nullptr, 0);
      });
      if (info) info->fallbacks = fallbacks;
      if (e) return info_done(info, e, c.launches, t0);
    }
  }
  if ((e = copy_R_out(Rdev, ncols, R, ldr, st))) return info_done(info, e, c.launches, t0);
  e = finish_status(ar, st, info);
  return info_done(info, e, c.launches, t0);
}

int rbo_block_orth_one_stage(rbo_sketch sk, int64_t n, int32_t ncols, int32_t s, double* V,
                             int64_t ldv, double* R, int64_t ldr, const rbo_opts* opts,
                             rbo_info* info, void* stream) {
  const int intra = opts ? opts->intra : RBO_INTRA_RANDCHOLQR;
  if (intra != RBO_INTRA_RANDCHOLQR && intra != RBO_INTRA_CHOLQR2) return RBO_ERR_ARG;
  return block_orth_impl(sk, n, ncols, s, s, V, ldv, R, ldr, opts, info, stream, 0, intra);
}

int rbo_block_orth_two_stage(rbo_sketch sk, int64_t n, int32_t ncols, int32_t s, int32_t s_hat,
                             double* V, int64_t ldv, double* R, int64_t ldr, const rbo_opts* opts,
                             rbo_info* info, void* stream) {
  return block_orth_impl(sk, n, ncols, s, s_hat, V, ldv, R, ldr, opts, info, stream, 1,
                         RBO_INTRA_RANDCHOLQR);
}

int rbo_block_orth_cholqr2(int64_t n, int32_t ncols, int32_t s, double* V, int64_t ldv, double* R,
                           int64_t ldr, const rbo_opts* opts, rbo_info* info, void* stream) {
  rbo_opts o = opts ? *opts : rbo_opts{};
  o.intra = RBO_INTRA_CHOLQR2;
  o.precision = RBO_PREC_FP64;
  return block_orth_impl(nullptr, n, ncols, s, s, V, ldv, R, ldr, &o, info, stream, 0,
                         RBO_INTRA_CHOLQR2);
}

int rbo_mpk_csr(const rbo_csr* A, const double* dscale, int32_t s, const double* v0, double* V,
                int64_t ldv, void* stream) {
  if (!A || A->n < 1 || !A->rowptr || !A->col || !A->val || A->nnz < 0 || A->nnz >= (1LL << 31) ||
      s < 1 || !v0 || !V || ldv < A->n)
    return RBO_ERR_ARG;
  int e = check_device();
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  Arena* ar = nullptr;
  if ((e = arena_prepare(&ar, 0))) return e;
  if (cudaMemsetAsync(ar->base, 0, 1024, st) != cudaSuccess) return RBO_ERR_CUDA;
  CsrDev M{A->n, A->nnz, A->rowptr, A->col, A->val};
  const double* prev = v0;
  for (int i = 0; i < s; ++i) {
    double* out = V + (int64_t)i * ldv;
    if ((e = spmv_launch(M, dscale, prev, out, ar->status, st))) return e;
    prev = out;
  }
  return finish_status(ar, st, nullptr);
}

}  // extern "C"

// CSR sparse kernels of the matrix-powers kernel (Section 4) and the small vector
// kernels of the GMRES driver.
//
// SpMV: rows of up to ~12 entries on average (stencils) go to a persistent kernel in
// which each warp stages the entries of 32 consecutive rows in shared memory and
// every lane runs its own row; denser rows use a group of LPR = 8 or 32 lanes per
// row that read consecutive entries and combine with shuffles in a fixed order.
// Every sum has a fixed order, so the result is deterministic.  The optional
// diagonal scaling D of the right Jacobi preconditioner (A D x) is applied to the
// gathered x entries; the optional shift terms of the Newton and Chebyshev bases
// are added to each output row.
#include <algorithm>
#include <vector>

#include "device_common.cuh"

namespace rbo {

// (A x)_r + a u_r + b uprev_r, in the order of the separate shift pass
__device__ __forceinline__ double shifted(double s, const SpmvShift& sh, int64_t r) {
  if (!sh.u) return s;
  double v = fma(sh.a, sh.u[r], s);
  if (sh.uprev) v = fma(sh.b, sh.uprev[r], v);
  return v;
}

// Entries with a column index outside [0, n), or rows whose pointers leave [0, nnz],
// are skipped and reported through the status word (RBO_ERR_ARG) instead of being
// dereferenced.
template <int LPR>
__global__ void __launch_bounds__(256) spmv_kernel(int64_t n, int64_t nnz,
                                                   const int32_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col,
                                                   const double* __restrict__ val,
                                                   const double* __restrict__ dscale,
                                                   const double* __restrict__ x,
                                                   const double* __restrict__ bvec,
                                                   double* __restrict__ y, DevStatus* status,
                                                   SpmvShift sh) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gid / LPR;
  const int sub = (int)(gid % LPR);
  double s = 0.0;
  if (row < n) {
    int beg = __ldg(rowptr + row), end = __ldg(rowptr + row + 1);
    if (beg < 0 || end < beg || (int64_t)end > nnz) {
      if (status && sub == 0) set_error(status, RBO_ERR_ARG, 11);
      end = beg;
    }
      for (int j = beg + sub; j < end; j += LPR) {
        const int cj = __ldg(col + j);
        if (cj < 0 || (int64_t)cj >= n) {
          if (status) set_error(status, RBO_ERR_ARG, 12);
          continue;
        }
        const double xv = dscale ? __ldg(dscale + cj) * __ldg(x + cj) : __ldg(x + cj);
        s = fma(__ldg(val + j), xv, s);
      }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, LPR);
  if (row < n && sub == 0) y[row] = bvec ? (bvec[row] - s) : shifted(s, sh, row);
}


// Short rows: each warp takes groups of 32 consecutive rows (persistent grid of 4
// blocks per SM; the row pointers of the warp's next group are loaded while the
// current group is processed).  The warp stages the entries of its rows in chunks of
// SCH (coalesced index and value loads, the x gathers issued by the same lanes), then
// every lane runs the multiply-adds of its own row from shared memory, as two
// interleaved chains (even and odd entries) added at the end.  No cross-lane float64
// reduction is needed: each float64 operation costs a slot of this GPU's narrow
// float64 pipe.
constexpr int SCH = 256;
__global__ void __launch_bounds__(256) spmv_stream_kernel(int64_t n, int64_t nnz,
                                                          const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const double* __restrict__ val,
                                                          const double* __restrict__ dscale,
                                                          const double* __restrict__ x,
                                                          const double* __restrict__ bvec,
                                                          double* __restrict__ y, DevStatus* status,
                                                          SpmvShift sh) {
  __shared__ double sv[8][SCH], sx[8][SCH];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ngroups = (n + 31) / 32;
  const int64_t gstride = (int64_t)gridDim.x * 8;
  int64_t g = (int64_t)blockIdx.x * 8 + warp;
  int beg = 0, end = 0;
  if (g < ngroups && g * 32 + lane < n) {
    beg = __ldg(rowptr + g * 32 + lane);
    end = __ldg(rowptr + g * 32 + lane + 1);
  }
  for (; g < ngroups; g += gstride) {
    // row pointers of this warp's next group, in flight during this group
    const int64_t gn = g + gstride;
    int nbeg = 0, nend = 0;
    if (gn < ngroups && gn * 32 + lane < n) {
      nbeg = __ldg(rowptr + gn * 32 + lane);
      nend = __ldg(rowptr + gn * 32 + lane + 1);
    }
    const int64_t r0 = g * 32, r = r0 + lane;
    const int nr = (int)((n - r0) < 32 ? (n - r0) : 32);
    const int e0 = __shfl_sync(0xffffffffu, beg, 0);
    const int e1 = __shfl_sync(0xffffffffu, end, nr - 1);
    const bool range_ok = e0 >= 0 && e1 >= e0 && (int64_t)e1 <= nnz;
    if (r < n && (!range_ok || beg < e0 || end < beg || end > e1)) {
      if (status) set_error(status, RBO_ERR_ARG, 11);
      end = beg;
    }
    double s = 0.0, s2 = 0.0;
    if (range_ok) {
      for (int c0 = e0; c0 < e1; c0 += SCH) {
        const int cn = (e1 - c0) < SCH ? (e1 - c0) : SCH;
        int cj[SCH / 32];
        double v[SCH / 32], xv[SCH / 32];
#pragma unroll
        for (int u = 0; u < SCH / 32; ++u) {
          const int t = u * 32 + lane;
          cj[u] = -1;
          v[u] = 0.0;
          if (t < cn) {
            cj[u] = __ldg(col + c0 + t);
            v[u] = __ldg(val + c0 + t);
          }
        }
#pragma unroll
        for (int u = 0; u < SCH / 32; ++u) {
          const int t = u * 32 + lane;
          xv[u] = 0.0;
          if (t < cn) {
            if (cj[u] < 0 || (int64_t)cj[u] >= n) {
              if (status) set_error(status, RBO_ERR_ARG, 12);
              v[u] = 0.0;
            } else {
              xv[u] = dscale ? __ldg(dscale + cj[u]) * __ldg(x + cj[u]) : __ldg(x + cj[u]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < SCH / 32; ++u) {
          const int t = u * 32 + lane;
          if (t < cn) {
            sv[warp][t] = v[u];
            sx[warp][t] = xv[u];
          }
        }
        __syncwarp();
        const int lo = beg > c0 ? beg : c0, hi = end < c0 + cn ? end : c0 + cn;
        int e = lo;
        for (; e + 1 < hi; e += 2) {
          s = fma(sv[warp][e - c0], sx[warp][e - c0], s);
          s2 = fma(sv[warp][e + 1 - c0], sx[warp][e + 1 - c0], s2);
        }
        if (e < hi) s = fma(sv[warp][e - c0], sx[warp][e - c0], s);
        __syncwarp();
      }
    }
    s += s2;
    if (r < n) y[r] = bvec ? (bvec[r] - s) : shifted(s, sh, r);
    beg = nbeg;
    end = nend;
  }
}

static int spmv_dispatch_inner(const CsrDev& A, const double* dscale, const double* x,
                               const double* b, double* y, DevStatus* status, cudaStream_t st,
                               const SpmvShift& sh);

template <int LPR>
static void spmv_go(const CsrDev& A, const double* dscale, const double* x, const double* b,
                    double* y, DevStatus* status, cudaStream_t st, const SpmvShift& sh) {
  const int64_t threads = A.n * LPR;
  const int64_t blocks = (threads + 255) / 256;
  spmv_kernel<LPR><<<(unsigned)blocks, 256, 0, st>>>(A.n, A.nnz, A.rowptr, A.col, A.val, dscale, x,
                                                     b, y, status, sh);
}

static int spmv_dispatch(const CsrDev& A, const double* dscale, const double* x, const double* b,
                         double* y, DevStatus* status, cudaStream_t st, const SpmvShift& sh) {
  if (A.n <= 0) return RBO_OK;
  SpmvShift k = sh;
  if (!k.u || b) k = SpmvShift();  // (a residual has no shift)
  if (k.b == 0.0) k.uprev = nullptr;
  ProfToken tok = prof_start(st);
  int e = spmv_dispatch_inner(A, dscale, x, b, y, status, st, k);
  // algorithmic bytes: values + column indices + row pointers, x and y once each
  // (plus b, the scaling vector and the shift's vectors when used); 2 flops per
  // stored entry (+2 per row and shift term)
  const double nn = (double)A.n, nz = (double)A.nnz;
  const int terms = (k.u ? 1 : 0) + (k.uprev ? 1 : 0);
  prof_stop(tok, st, 1, 12.0 * nz + 4.0 * (nn + 1) + 16.0 * nn + (b ? 8.0 * nn : 0.0) +
                            (dscale ? 8.0 * nn : 0.0) + 8.0 * terms * nn,
            2.0 * nz + 2.0 * terms * nn);
  return e;
}

static int spmv_dispatch_inner(const CsrDev& A, const double* dscale, const double* x,
                               const double* b, double* y, DevStatus* status, cudaStream_t st,
                               const SpmvShift& sh) {
  const double avg = A.n > 0 ? (double)A.nnz / (double)A.n : 0.0;
  if (avg <= 12.0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = std::min<int64_t>((A.n + 255) / 256, (int64_t)std::max(sms, 1) * 4);
    spmv_stream_kernel<<<(unsigned)blocks, 256, 0, st>>>(A.n, A.nnz, A.rowptr, A.col, A.val, dscale,
                                                          x, b, y, status, sh);
  } else if (avg <= 24.0)
    spmv_go<8>(A, dscale, x, b, y, status, st, sh);
  else
    spmv_go<32>(A, dscale, x, b, y, status, st, sh);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

int spmv_launch(const CsrDev& A, const double* dscale, const double* x, double* y, DevStatus* status,
                cudaStream_t st, const SpmvShift& sh) {
  return spmv_dispatch(A, dscale, x, nullptr, y, status, st, sh);
}

int residual_launch(const CsrDev& A, const double* b, const double* x, double* r, DevStatus* status,
                    cudaStream_t st) {
  return spmv_dispatch(A, nullptr, x, b, r, status, st, SpmvShift());
}

__global__ void scale_columns_kernel(int64_t n, int64_t nnz, const int32_t* __restrict__ col,
                                     const double* __restrict__ val, const double* __restrict__ ds,
                                     double* __restrict__ out) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; j < nnz; j += stride) {
    const int32_t c = col[j];
    out[j] = (c >= 0 && (int64_t)c < n) ? val[j] * ds[c] : 0.0;
  }
}

int scale_columns_launch(const CsrDev& A, const double* dscale, double* val_out, cudaStream_t st) {
  if (A.nnz <= 0) return RBO_OK;
  int64_t blocks = std::min<int64_t>((A.nnz + 255) / 256, 65535LL * 16);
  scale_columns_kernel<<<(unsigned)blocks, 256, 0, st>>>(A.n, A.nnz, A.col, A.val, dscale, val_out);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

__global__ void jacobi_kernel(int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, const double* __restrict__ val,
                              double* __restrict__ ds, DevStatus* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double dia = 0.0;
  int beg = rowptr[i], end = rowptr[i + 1];
  if (beg < 0 || end < beg || (int64_t)end > nnz) end = beg;
  for (int j = beg; j < end; ++j)
    if (col[j] == (int32_t)i) dia = val[j];
  if (dia == 0.0) {
    set_error(status, RBO_ERR_ARG, 10);
    ds[i] = 0.0;
  } else {
    ds[i] = 1.0 / dia;
  }
}

int jacobi_launch(const CsrDev& A, double* dscale, DevStatus* status, cudaStream_t st) {
  if (A.n <= 0) return RBO_OK;
  jacobi_kernel<<<(unsigned)((A.n + 255) / 256), 256, 0, st>>>(A.n, A.nnz, A.rowptr, A.col, A.val, dscale,
                                                                status);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

// y = Q z (accumulate = 0) or y += Q z: one thread per row, z in shared memory
__global__ void gemv_update_kernel(int64_t n, int k, const double* __restrict__ Q, int64_t ldq,
                                   const double* __restrict__ z, double* __restrict__ y,
                                   int accumulate) {
  __shared__ double zs[256];
  for (int t = threadIdx.x; t < k; t += blockDim.x) zs[t] = z[t];
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int c = 0; c < k; ++c) s = fma(Q[i + c * ldq], zs[c], s);
  y[i] = accumulate ? y[i] + s : s;
}

// x += D t  (D = diag(ds), or the identity when ds is null)
__global__ void axpy_scaled_kernel(int64_t n, const double* __restrict__ ds,
                                   const double* __restrict__ t, double* __restrict__ x) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] += ds ? ds[i] * t[i] : t[i];
}

int axpy_scaled_launch(int64_t n, const double* ds, const double* t, double* x, cudaStream_t st) {
  if (n <= 0) return RBO_OK;
  axpy_scaled_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, ds, t, x);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

// Newton-basis step: out += a u + b uprev (uprev may be null when b = 0)
int gemv_update_launch(int64_t n, int k, const double* Q, int64_t ldq, const double* z, double* y,
                       int accumulate, cudaStream_t st) {
  if (n <= 0 || k <= 0) return RBO_OK;
  if (k > 256) return RBO_ERR_ARG;
  gemv_update_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, k, Q, ldq, z, y, accumulate);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

__global__ void scale_vec_kernel(int64_t n, const double* __restrict__ ds, const double* __restrict__ y,
                                 double* __restrict__ x, int mode) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = y[i];
  if (ds) v = mode == 0 ? v * ds[i] : v / ds[i];
  x[i] = v;
}

int scale_vec_launch(int64_t n, const double* dscale, const double* y, double* x, int mode,
                     cudaStream_t st) {
  if (n <= 0) return RBO_OK;
  scale_vec_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, dscale, y, x, mode);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

}  // namespace rbo

namespace rbo {

// ---- SELL-32: the short-row matrices of the MPK in sliced ELL form -------------------
// A warp owns a slice of 32 rows and a lane its row: slot j of the slice is one
// coalesced 256-byte value load and 128-byte index load for the whole warp, and the
// slots of a row are summed in two interleaved chains (even, odd j) added at the end, a
// fixed order.  Padding slots (value 0, the row's own index) cost a multiply-add.

__global__ void sell_width_kernel(int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                                  int32_t* __restrict__ width, DevStatus* status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t k = t >> 5;
  const int lane = (int)(t & 31);
  const int64_t nsl = (n + 31) / 32;
  if (k >= nsl) return;  // whole warps (nsl * 32 threads are launched)
  const int64_t r = k * 32 + lane;
  int len = 0;
  if (r < n) {
    const int beg = rowptr[r], end = rowptr[r + 1];
    if (beg < 0 || end < beg || (int64_t)end > nnz) {
      if (status) set_error(status, RBO_ERR_ARG, 11);
    } else {
      len = end - beg;
    }
  }
  len = __reduce_max_sync(0xffffffffu, len);
  if (lane == 0) width[k] = len;
}

__global__ void sell_fill_kernel(int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ ccol, const double* __restrict__ cval,
                                 const int64_t* __restrict__ soff, int32_t* __restrict__ col,
                                 double* __restrict__ val, DevStatus* status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t k = t >> 5;
  const int lane = (int)(t & 31);
  if (k >= (n + 31) / 32) return;
  const int64_t r = k * 32 + lane;
  const int64_t off = soff[k];
  const int w = (int)((soff[k + 1] - off) / 32);
  int beg = 0, len = 0;
  if (r < n) {
    beg = rowptr[r];
    const int end = rowptr[r + 1];
    if (beg >= 0 && end >= beg && (int64_t)end <= nnz) len = end - beg;
  }
  const int32_t self = (int32_t)(r < n ? r : 0);
  for (int j = 0; j < w; ++j) {
    int32_t c = self;
    double v = 0.0;
    if (j < len) {
      const int32_t cj = ccol[beg + j];
      if (cj < 0 || (int64_t)cj >= n) {
        if (status) set_error(status, RBO_ERR_ARG, 12);
      } else {
        c = cj;
        v = cval[beg + j];
      }
    }
    col[off + (int64_t)j * 32 + lane] = c;
    val[off + (int64_t)j * 32 + lane] = v;
  }
}

__global__ void __launch_bounds__(256, 6) spmv_sell_kernel(int64_t n, int64_t nsl, const int64_t* __restrict__ soff,
                                                           const int32_t* __restrict__ col,
                                                           const double* __restrict__ val,
                                                           const double* __restrict__ x, double* __restrict__ y,
                                                           SpmvShift sh) {
  // one slice per warp (the grid covers the matrix): every warp's loads are in flight
  // at once; slices of up to 8 slots load all indices and values before the gathers
  const int lane = threadIdx.x & 31;
  const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= nsl) return;
  const int64_t off = __ldg(soff + k);
  const int w = (int)((__ldg(soff + k + 1) - off) >> 5);
  const int32_t* cp = col + off + lane;
  const double* vp = val + off + lane;
  double s0 = 0.0, s1 = 0.0;
  if (w <= 8) {
    int32_t c[8];
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = j < w ? __ldg(cp + 32 * j) : 0;
      v[j] = j < w ? __ldg(vp + 32 * j) : 0.0;
    }
    double xv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) xv[j] = j < w ? __ldg(x + c[j]) : 0.0;
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      if (j < w) s0 = fma(v[j], xv[j], s0);
      if (j + 1 < w) s1 = fma(v[j + 1], xv[j + 1], s1);
    }
  } else {
    for (int j = 0; j < w; ++j) {
      const double vv = __ldg(vp + 32 * j), xx = __ldg(x + __ldg(cp + 32 * j));
      if (j & 1) s1 = fma(vv, xx, s1);
      else s0 = fma(vv, xx, s0);
    }
  }
  const int64_t r = k * 32 + lane;
  if (r < n) y[r] = shifted(s0 + s1, sh, r);
}

}  // namespace rbo

namespace rbo {

int sell_build(const CsrDev& A, int64_t cap_slots, int64_t* soff, int32_t* width, int32_t* col,
               double* val, DevStatus* status, cudaStream_t st, SellDev* out) {
  *out = SellDev();
  if (A.n <= 0) return RBO_OK;
  const int64_t nsl = (A.n + 31) / 32;
  const int64_t threads = nsl * 32;
  sell_width_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A.n, A.nnz, A.rowptr, width, status);
  if (cudaGetLastError() != cudaSuccess) return RBO_ERR_CUDA;
  std::vector<int32_t> wh((size_t)nsl);
  std::vector<int64_t> oh((size_t)nsl + 1);
  if (cudaMemcpyAsync(wh.data(), width, (size_t)nsl * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RBO_ERR_CUDA;
  oh[0] = 0;
  for (int64_t k = 0; k < nsl; ++k) oh[(size_t)k + 1] = oh[(size_t)k] + 32 * (int64_t)wh[(size_t)k];
  if (oh[(size_t)nsl] > cap_slots) return RBO_OK;  // too much padding: stay with CSR
  if (cudaMemcpyAsync(soff, oh.data(), (size_t)(nsl + 1) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return RBO_ERR_CUDA;
  sell_fill_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A.n, A.nnz, A.rowptr, A.col, A.val, soff,
                                                                      col, val, status);
  if (cudaGetLastError() != cudaSuccess) return RBO_ERR_CUDA;
  // the host copy of the offsets must outlive the asynchronous upload
  if (cudaStreamSynchronize(st) != cudaSuccess) return RBO_ERR_CUDA;
  out->n = A.n;
  out->nslices = nsl;
  out->soff = soff;
  out->col = col;
  out->val = val;
  return RBO_OK;
}

int spmv_sell_launch(const SellDev& S, int64_t nnz, const double* x, double* y, cudaStream_t st,
                     const SpmvShift& sh) {
  if (S.n <= 0) return RBO_OK;
  SpmvShift k = sh;
  if (!k.u) k = SpmvShift();
  if (k.b == 0.0) k.uprev = nullptr;
  const int64_t blocks = (S.nslices + 7) / 8;
  if (blocks > 0x7FFFFFFFLL) return RBO_ERR_ARG;
  ProfToken tok = prof_start(st);
  spmv_sell_kernel<<<(unsigned)blocks, 256, 0, st>>>(S.n, S.nslices, S.soff, S.col, S.val, x, y, k);
  // algorithmic bytes and flops as for the CSR kernel (the stored entries, not the padding)
  const double nn = (double)S.n, nz = (double)nnz;
  const int terms = (k.u ? 1 : 0) + (k.uprev ? 1 : 0);
  prof_stop(tok, st, 1, 12.0 * nz + 4.0 * (nn + 1) + 16.0 * nn + 8.0 * terms * nn, 2.0 * nz + 2.0 * terms * nn);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

}  // namespace rbo

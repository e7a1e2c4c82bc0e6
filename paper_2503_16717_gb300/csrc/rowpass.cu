// The row pass: one fused streaming pass over the rows of a tall-skinny panel.
//
// Every step of the block orthogonalization that touches n-row data is a row pass
// (BCGS Gram and update, sketch apply, the TRSMs of CholQR/RandHH, the forward
// substitution of RandBCGS2 and the Gram matrices feeding the Cholesky
// factorisations; Sections 4-7 of the paper):
//
//   per row r:   y'_r = (y_r - x_r C) Tri^{-1}      (or y_r Tri^{-1} - x_r C)
//                write y'_r back to Y                     (optional)
//                Z   += [x_r, y'_r]^T y'_r                (X^T Y' and/or Y'^T Y')
//                SK  += s_r y'_r  (sketch column s_r: zeta entries +-1, hashed)
//
// This file holds the kernel of the passes without a scattered sketch (Gram and
// transform passes) and the launcher of all row passes; the sketch passes run in
// rowpass_sk.cu, the tensor-core Gram in ozaki.cu.
//
// Row tiles of T rows are staged in shared memory by the bulk-copy (TMA) engine
// (cp.async.bulk + mbarrier, double buffered; ragged tiles use plain loads).
// Each CTA owns a fixed set of tiles, keeps its partial Z in registers (one
// output per thread slot), then writes one partial.  A two-level ticketed tree
// (groups of 16 CTAs, then one top reducer) sums the partials in a fixed order, so
// results are bitwise reproducible; the last CTA runs the small dense epilogue
// (Cholesky, Householder, sketched BCGS2-HH, R assembly) on the reduced values.
#include <algorithm>
#include <map>
#include <mutex>

#include "rowpass_common.cuh"

namespace rbo {

// ------------------------------------------------------------------------------------
// Gram task bodies: one Z row against CW columns of Y' (a register block), over the
// tile rows g, g + tpo, ...  CW is a compile-time constant so that a narrow last
// block (b not a multiple of CB) issues no masked-off float64 instructions.
// ------------------------------------------------------------------------------------
template <int CW>
__device__ __forceinline__ void gram_rows_f64(double (&acc)[CB], const double* z, const double* y,
                                              int g, int T, int tpo, int TP) {
  for (int rr = g; rr < T; rr += tpo) {
    const double zv = z[rr];
#pragma unroll
    for (int c = 0; c < CW; ++c) acc[c] = fma(zv, y[(size_t)c * TP + rr], acc[c]);
  }
}
// float32 values in the first 4 bytes of each 8-byte slot
template <int CW>
__device__ __forceinline__ void gram_rows_f32(float (&acc)[CB], const double* z, const double* y,
                                              int g, int T, int tpo, int TP) {
  for (int rr = g; rr < T; rr += tpo) {
    const float zv = reinterpret_cast<const float*>(z + rr)[0];
#pragma unroll
    for (int c = 0; c < CW; ++c)
      acc[c] = fmaf(zv, reinterpret_cast<const float*>(y + (size_t)c * TP + rr)[0], acc[c]);
  }
}
template <int CW>
__device__ __forceinline__ void gram_rows_df(df (&acc)[CB], const df* z, const df* y, int g, int T,
                                             int tpo, int TP) {
  for (int rr = g; rr < T; rr += tpo) {
    const df zv = z[rr];
#pragma unroll
    for (int c = 0; c < CW; ++c) df_fma_acc(acc[c], zv, y[(size_t)c * TP + rr]);
  }
}
// ------------------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------------------
template <int ARITH>
__global__ void __launch_bounds__(NT, (ARITH == 0 ? 3 : 2)) rowpass_kernel(const __grid_constant__ PassDev P) {
  // ARITH 0: float64; 1: float32 for X^T Y' (mixed precision); 2: float32 pairs for
  // the transform and the Gram.  Passes that scatter a sparse sketch run in
  // rowpass_sk_kernel (rowpass_sk.cu).
  constexpr bool MIXED = ARITH == 1;
  constexpr bool DF = ARITH == 2;
  constexpr int IPTA = DF ? 2 : IPT;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ int s_last;
  const RowPass& rp = P.p;
  if (read_code(P.status) != 0) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = P.T, TP = P.TP, a = rp.a, b = rp.b;
  // Z rows: Gaussian sketch rows, then X rows (acc_x), then Y' rows (acc_y)
  const int gd = rp.sk_gd;
  const int ax = gd + (rp.acc_x ? a : 0);
  const int64_t n = rp.n;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  double* Cs = reinterpret_cast<double*>(smem + P.off_c);
  double* Ts = reinterpret_cast<double*>(smem + P.off_tri);
  double* dinv = reinterpret_cast<double*>(smem + P.off_dinv);
  double* gth = reinterpret_cast<double*>(smem + P.off_gth);  // Gaussian sketch tile

  // small matrices + sketch copies
  if (rp.C) {
    const int ldc = rp.ldc > 0 ? rp.ldc : a;
    for (int t = tid; t < a * b; t += NT) {
      const double v = rp.C[(t % a) + (size_t)(t / a) * ldc];
      if (DF && rp.small_coeffs && !rp.Tri)
        reinterpret_cast<df*>(Cs)[t] = df_from_double(v);
      else
        Cs[t] = v;
    }
  }
  if (rp.Tri) {
    const int ldt = rp.ldtri > 0 ? rp.ldtri : b;
    for (int t = tid; t < b * b; t += NT) {
      const int i = t % b, c = t / b;
      Ts[t] = (i <= c) ? rp.Tri[i + (size_t)c * ldt] : 0.0;
    }
    for (int t = tid; t < b; t += NT) dinv[t] = 1.0 / rp.Tri[t + (size_t)t * ldt];
  }
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // Z tasks: item = (Z row i, block of up to CB columns), split over `tpo` row
  // subsets; thread t owns tasks t, t + NT, ... (at most IPT)
  double acc[IPTA][CB];
  float accf[IPTA][CB];
  df acci[IPTA][CB];  // float-pair partial sums, flushed into acc every few tiles
#pragma unroll
  for (int k = 0; k < IPTA; ++k)
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      acc[k][c] = 0.0;
      accf[k][c] = 0.0f;
      acci[k][c] = df{0.f, 0.f};
    }
  int since_flush = 0;
  auto flush = [&]() {
#pragma unroll
    for (int k = 0; k < IPTA; ++k)
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        acc[k][c] += df_to_double_fast(acci[k][c]);
        acci[k][c] = df{0.f, 0.f};
      }
  };
  // float-pair arithmetic: the projection only when its coefficients are small
  // (re-orthogonalization, whose subtrahend is O(eps kappa) of the data), so that the
  // 48-bit rounding cannot reach the backward error; triangular solves and
  // large-coefficient projections stay float64; Gram sums always in pairs
  const bool df_pre = DF && !rp.Tri && rp.C && rp.small_coeffs;
  const bool df_post = DF && P.no > 0 && !df_pre;

  const int ncol_tile = (a + b);
  auto stage_X = [&](int s) {
    return reinterpret_cast<double*>(smem + P.off_stage + (size_t)s * P.stage_bytes);
  };
  auto stage_Y = [&](int s) { return stage_X(s) + (size_t)a * TP; };

  // bulk-copy a full tile into stage s (all lanes of warp 0: one copy per lane)
  auto issue_tile = [&](int tile, int s) {
    const int64_t r0 = (int64_t)tile * T;
    double* xs = stage_X(s);
    double* ys = stage_Y(s);
    const uint32_t bytes = (uint32_t)T * 8u;
    if (lane == 0) mbar_arrive_expect_tx(&bars[s], bytes * (uint32_t)ncol_tile);
    __syncwarp();
    for (int j = lane; j < a + b; j += 32) {
      if (j < a)
        bulk_copy_g2s(xs + (size_t)j * TP, rp.X + j * rp.ldx + r0, bytes, &bars[s]);
      else
        bulk_copy_g2s(ys + (size_t)(j - a) * TP, rp.Y + (j - a) * rp.ldy + r0, bytes, &bars[s]);
    }
  };
  auto bulk_ok = [&](int tile) {
    return P.use_bulk && ((int64_t)(tile + 1) * T <= n);
  };

  uint32_t phase[NST] = {0u, 0u};
  int first = blockIdx.x;
  if (first < P.ntiles && bulk_ok(first) && warp == 0) issue_tile(first, 0);

  int it = 0;
  bool timed_out = false;
  for (int tile = first; tile < P.ntiles; tile += gridDim.x, ++it) {
    const int s = it & 1;
    const int64_t r0 = (int64_t)tile * T;
    const int rows = (n - r0 < (int64_t)T) ? (int)(n - r0) : T;
    double* xs = stage_X(s);
    double* ys = stage_Y(s);
    if (bulk_ok(tile)) {
      if (!mbar_wait_bounded(&bars[s], phase[s])) {
        timed_out = true;
      }
      phase[s] ^= 1u;
    } else {
      // ragged or unaligned tile: plain coalesced loads with zero fill
      for (int t = tid; t < ncol_tile * T; t += NT) {
        int col = t / T, r = t % T;
        double v = 0.0;
        if (r < rows) v = (col < a) ? rp.X[col * rp.ldx + r0 + r] : rp.Y[(col - a) * rp.ldy + r0 + r];
        xs[(size_t)col * TP + r] = v;  // X and Y stages are contiguous
      }
      __syncthreads();
    }
    if (timed_out) {
      if (tid == 0) set_error(P.status, RBO_ERR_TIMEOUT, 1);
      return;
    }
    // prefetch the next tile of this CTA into the other stage
    const int nxt = tile + gridDim.x;
    if (warp == 0 && nxt < P.ntiles && bulk_ok(nxt)) {
      fence_proxy_async();
      issue_tile(nxt, s ^ 1);
    }

    // float64 -> float pairs in place (8 bytes each), integer operations only
    auto to_pairs = [&]() {
      for (int t = tid; t < ncol_tile * T; t += NT) {
        const size_t e = (size_t)(t / T) * TP + (t % T);
        reinterpret_cast<df*>(xs)[e] = df_from_double(xs[e]);
      }
      __syncthreads();
    };
    if (df_pre) to_pairs();

    // Gaussian sketch entries of the tile's rows (float32 Box-Muller; zero past n),
    // as extra Z rows of the Gram phase: S Y' = sum over rows of theta_r y'_r^T
    if (gd > 0) {
      for (int t = tid; t < gd * T; t += NT) {
        const int r = t % T, k = t / T;
        const float v = r < rows ? gauss_entry(rp.sk_seed, (uint64_t)(r0 + r), k, gd) : 0.0f;
        if (MIXED)
          reinterpret_cast<float*>(gth + (size_t)k * TP + r)[0] = v;
        else
          gth[(size_t)k * TP + r] = (double)v;
      }
      __syncthreads();
    }

    // ---- phase A: y' = transform(y), in place in the Y stage --------------------
    // y' = y Tri^-1 by rows, in column blocks of CB: the block's update by the
    // finished columns runs over all (row, column) pairs, the substitution inside the
    // block over rows.  Each entry subtracts its terms in column order, as an
    // unblocked row-by-row substitution would.
    auto tri_solve = [&]() {
      for (int c0 = 0; c0 < b; c0 += CB) {
        const int cw = min(CB, b - c0);
        if (c0 > 0) {
          for (int t = tid; t < T * cw; t += NT) {
            const int r = t % T, c = c0 + t / T;
            double v = ys[c * TP + r];
            for (int i = 0; i < c0; ++i) v = fma(-ys[i * TP + r], Ts[i + c * b], v);
            ys[c * TP + r] = v;
          }
          __syncthreads();
        }
        for (int r = tid; r < T; r += NT) {
          for (int c = c0; c < c0 + cw; ++c) {
            double v = ys[c * TP + r];
            for (int i = c0; i < c; ++i) v = fma(-ys[i * TP + r], Ts[i + c * b], v);
            ys[c * TP + r] = v * dinv[c];
          }
        }
        if (c0 + CB < b) __syncthreads();
      }
    };
    auto project = [&]() {
      if (df_pre) {
        df* yp = reinterpret_cast<df*>(ys);
        const df* xp = reinterpret_cast<const df*>(xs);
        const df* cp = reinterpret_cast<const df*>(Cs);
        for (int t = tid; t < T * b; t += NT) {
          const int r = t % T, c = t / T;
          const df* cc = cp + (size_t)c * a;
          df v = yp[c * TP + r];
          for (int i = 0; i < a; ++i) df_fma_acc(v, df_neg(xp[i * TP + r]), cc[i]);
          yp[c * TP + r] = df_norm(v);
        }
        return;
      }
      // one (row, column) element per task; two interleaved partial sums
      for (int t = tid; t < T * b; t += NT) {
        const int r = t % T, c = t / T;
        const double* cc = Cs + (size_t)c * a;
        double v0 = ys[c * TP + r], v1 = 0.0;
        int i = 0;
        for (; i + 1 < a; i += 2) {
          v0 = fma(-xs[i * TP + r], cc[i], v0);
          v1 = fma(-xs[(i + 1) * TP + r], cc[i + 1], v1);
        }
        if (i < a) v0 = fma(-xs[i * TP + r], cc[i], v0);
        ys[c * TP + r] = v0 + v1;
      }
    };
    if (rp.Tri && rp.tri_first) {
      tri_solve();
      __syncthreads();
    }
    if (rp.C) {
      project();
      __syncthreads();
    }
    if (rp.Tri && !rp.tri_first) {
      tri_solve();
      __syncthreads();
    }
    if (rp.write_y) {
      for (int t = tid; t < b * T; t += NT) {
        int c = t / T, rr = t % T;
        if (df_pre) {
          const size_t e = (size_t)c * TP + rr;
          const double v = df_to_double_fast(reinterpret_cast<const df*>(ys)[e]);
          if (rr < rows) rp.Y[c * rp.ldy + r0 + rr] = v;
        } else {
          if (rr < rows) rp.Y[c * rp.ldy + r0 + rr] = ys[(size_t)c * TP + rr];
        }
      }
    }
    if (df_post) {
      __syncthreads();  // float64 values of the tile consumed by the write-back
      to_pairs();
    }

    // ---- phase B: Gram outputs Z = [X, Y']^T Y' --------------------------------
    if (MIXED && P.no > 0) {
      // float32 copies of the tile (integer-ALU conversion) in place: the float for
      // element t sits in the first 4 bytes of its double slot
      __syncthreads();
      for (int t = tid; t < ncol_tile * T; t += NT) {
        const size_t e = (size_t)(t / T) * TP + (t % T);
        float f = f64_to_f32_int(xs[e]);
        reinterpret_cast<float*>(xs + e)[0] = f;
      }
      __syncthreads();
    }
    if (DF && P.no > 0) {
#pragma unroll
      for (int k = 0; k < IPTA; ++k) {
        const int task = tid + k * NT;
        if (task < P.tasks) {
          const int item = task % P.items, g = task / P.items;
          int blk = 0;
          while (blk + 1 < P.nblk && item >= P.blk_start[blk + 1]) ++blk;
          const int i = item - P.blk_start[blk], c0 = min(blk * P.cw, b - P.cw);
          const int cw = P.cw;
          const df* zsrc = reinterpret_cast<const df*>((i < ax) ? xs + (size_t)(i - gd) * TP
                                                                 : ys + (size_t)(i - ax) * TP);
          const df* ysrc = reinterpret_cast<const df*>(ys + (size_t)c0 * TP);
          RBO_CW_DISPATCH(gram_rows_df, cw, acci[k], zsrc, ysrc, g, T, P.tpo, TP)
        }
      }
      if (++since_flush >= P.flush_tiles) {
        flush();
        since_flush = 0;
      }
    } else if (P.no > 0) {
#pragma unroll
      for (int k = 0; k < IPTA; ++k) {
        const int task = tid + k * NT;
        if (task < P.tasks) {
          const int item = task % P.items, g = task / P.items;
          int blk = 0;
          while (blk + 1 < P.nblk && item >= P.blk_start[blk + 1]) ++blk;
          const int i = item - P.blk_start[blk], c0 = min(blk * P.cw, b - P.cw);
          const int cw = P.cw;
          const double* zsrc = (i < gd)   ? gth + (size_t)i * TP
                               : (i < ax) ? xs + (size_t)(i - gd) * TP
                                          : ys + (size_t)(i - ax) * TP;
          const double* ysrc = ys + (size_t)c0 * TP;
          if (MIXED) {
            RBO_CW_DISPATCH(gram_rows_f32, cw, accf[k], zsrc, ysrc, g, T, P.tpo, TP)
          } else {
            RBO_CW_DISPATCH(gram_rows_f64, cw, acc[k], zsrc, ysrc, g, T, P.tpo, TP)
          }
        }
      }
    }
    __syncthreads();  // stage s free for reuse
  }

  // ---------------- partials + fixed-order two-level tree -------------------------
  if (P.L == 0) return;
  double* mypart = P.partials + (size_t)blockIdx.x * P.L;
  if (P.no > 0) {
    if (DF) flush();
    // combine the tpo row-subset partial sums of every item in a fixed order
    double* comb = reinterpret_cast<double*>(smem + P.off_stage);  // tasks x CB
#pragma unroll
    for (int k = 0; k < IPTA; ++k) {
      const int task = tid + k * NT;
      if (task < P.tasks)
#pragma unroll
        for (int c = 0; c < CB; ++c) comb[(size_t)task * CB + c] = MIXED ? (double)accf[k][c] : acc[k][c];
    }
    __syncthreads();
    for (int o = tid; o < P.no; o += NT) {
      const int i = o / b, c = o % b;
      // Y'^T Y' is symmetric: its entries below the diagonal come from the upper
      // triangle (the same products summed in the same order)
      int zi = i, zc = c;
      if (i >= ax && i - ax > c) {
        zi = ax + c;
        zc = i - ax;
      }
      const int blk = zc / P.cw, c0 = min(blk * P.cw, b - P.cw);
      const int item = P.blk_start[blk] + zi, cc = zc - c0;
      double sum = 0.0;
      for (int g = 0; g < P.tpo; ++g) sum += comb[(size_t)(g * P.items + item) * CB + cc];
      mypart[o] = sum;
    }
  }
  tree_reduce_epilogue(P, smem, &s_flag, &s_last);
}

// ------------------------------------------------------------------------------------
// host launcher
// ------------------------------------------------------------------------------------
// Per-device launch facts, cached on first use (guarded: calls for different devices
// may come from different host threads).
constexpr int MAX_DEV = 64;
static std::mutex g_launch_mu;
static int g_num_sms[MAX_DEV] = {};
static int g_smem_max[MAX_DEV][3] = {};
static std::map<long long, int> g_occ;

static int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) dev = 0;
  return dev;
}

static int sm_count() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_launch_mu);
  if (g_num_sms[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_num_sms[dev] = n > 0 ? n : 1;
  }
  return g_num_sms[dev];
}

// Largest dynamic shared memory of the row-pass kernel (opt-in limit minus its
// static shared memory); raises the kernel's limit to it on first use on a device.
template <int ARITH>
static int smem_limit_locked(int dev) {
  int& lim = g_smem_max[dev][ARITH];
  if (lim == 0) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    size_t stat = 0;
    if (cudaFuncGetAttributes(&fa, rowpass_kernel<ARITH>) == cudaSuccess) stat = fa.sharedSizeBytes;
    lim = optin - (int)stat - 64;
    if (cudaFuncSetAttribute(rowpass_kernel<ARITH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             lim) != cudaSuccess) {
      cudaGetLastError();
      lim = 48 * 1024 - (int)stat;
    }
  }
  return lim;
}

template <int ARITH>
static int smem_limit() {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_launch_mu);
  return smem_limit_locked<ARITH>(dev);
}

template <int ARITH>
static int occupancy(int smem) {
  const int dev = current_device();
  std::lock_guard<std::mutex> lk(g_launch_mu);
  const long long key = ((long long)dev << 40) | ((long long)smem * 4 + ARITH);
  auto it = g_occ.find(key);
  if (it != g_occ.end()) return it->second;
  int nb = 0;
  smem_limit_locked<ARITH>(dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rowpass_kernel<ARITH>, NT, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  if (nb < 1) nb = 1;
  g_occ[key] = nb;
  return nb;
}

int rowpass_launch(const RowPass& rpin, Arena* ar, cudaStream_t st, int* launches) {
  RowPass rp = rpin;
  if (rp.n <= 0 || rp.b <= 0 || rp.b > 64 || rp.a < 0 || rp.a > 128) return RBO_ERR_ARG;
  if (rp.a > 0 && rp.X == nullptr) return RBO_ERR_ARG;
  if (rp.a == 0) { rp.C = nullptr; rp.acc_x = 0; }
  // Gram passes of the tensor-core mode go to the digit-product kernel when their shape
  // allows it and (unless the caller asked for it outright, ozaki == 2) when it beats
  // the float64 pass (ozaki.cu); every other pass runs here in float64
  if (rp.ozaki && ozaki_gram_supported(rp) && (rp.ozaki == 2 || ozaki_gram_pays(rp)))
    return ozaki_gram_launch(rp, ar, st, launches, sm_count());
  if (rp.sk_d > DMAX || rp.sk_zeta > ZMAX) return RBO_ERR_ARG;
  if (rp.sk_gd < 0 || rp.sk_gd > 256 || rp.sk_cg < 0 || rp.sk_cg > DMAX) return RBO_ERR_ARG;
  if (rp.sk_gd > 0 && rp.sk_d > 0) return RBO_ERR_ARG;
  const int zr = rp.sk_gd + (rp.acc_x ? rp.a : 0) + (rp.acc_y ? rp.b : 0);
  const int no = zr * rp.b;
  if (no > 8192) return RBO_ERR_ARG;
  const int dsk = rp.sk_d > 0 ? rp.sk_d : 0;
  const int L = no + dsk * rp.b;
  // Z work split: items (Z row, block of CB columns), tpo row subsets per item
  // Z columns in nblk blocks of one width cw <= CB (the last block starts at b - cw
  // and may overlap its neighbour): every Gram task has the same trip counts
  const int nblk = (rp.b + CB - 1) / CB, cw = (rp.b + nblk - 1) / nblk;
  const int axr = rp.sk_gd + (rp.acc_x ? rp.a : 0);
  int blk_start[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int k = 0; k < nblk; ++k) {
    const int c0 = std::min(k * cw, rp.b - cw);
    blk_start[k + 1] = blk_start[k] + axr + (rp.acc_y ? std::min(rp.b, c0 + cw) : 0);
  }
  const int items = zr > 0 ? blk_start[nblk] : 0;
  if (items > IPT * NT) return RBO_ERR_ARG;
  // arithmetic: float32 pairs only where they apply (transform or Gram, no sketch
  // together with a Gram, at most 2 Gram tasks per thread); float64 otherwise
  int arith = rp.mixed ? 1 : 0;
  if (rp.df64 && !rp.mixed) {
    const bool pre = !rp.Tri && rp.C && rp.small_coeffs;
    const bool ok = (no > 0 || pre) && dsk == 0 && rp.sk_gd == 0 && items <= 2 * NT;
    arith = ok ? 2 : 0;
  }
  const int mixed = arith == 1 ? 1 : 0;
  if (dsk > 0) {
    // sketch passes run on the tiles of the call's sketch schedule, without a Gram
    if (no > 0) return RBO_ERR_ARG;
    if (rp.sk.rec == nullptr || rp.sk.mcap != sketch_sched_mcap(rp.sk.T, dsk, rp.sk_zeta) ||
        rp.sk.rec_bytes != sketch_sched_rec_bytes(rp.sk.T, dsk, rp.sk_zeta))
      return RBO_ERR_ARG;
    return rowpass_sk_launch(rp, ar, st, launches, sm_count(), L, mixed);
  }

  // tile height: the tallest tile up to 512 rows whose stage stays within STAGE_TARGET
  // bytes (narrow panels need tall tiles to keep enough bytes in flight), at least 64
  // rows, halved while the layout does not fit
  int T = 64;
  while (T < 512 && (size_t)(rp.a + rp.b) * (2 * T + 2) * 8 <= STAGE_TARGET) T *= 2;
  size_t smem = 0;
  int tpo = 1, tasks = 0;
  size_t off_stage = 0, stage_bytes = 0, off_c = 0, off_tri = 0, off_dinv = 0, off_red = 0,
         off_gth = 0;
  for (;;) {
    tpo = 1;
    if (items > 0)
      while (items * tpo * 2 <= NT && tpo * 2 <= T / 4) tpo *= 2;
    tasks = items * tpo;
    const int TP = T + 2;
    off_stage = 64;
    stage_bytes = (size_t)(rp.a + rp.b) * TP * 8;  // TP even: 16-byte multiple
    size_t o = off_stage + NST * stage_bytes;
    off_c = o; o += (rp.C ? (size_t)rp.a * rp.b * 8 : 0);
    off_tri = o; o += (rp.Tri ? (size_t)rp.b * rp.b * 8 : 0);
    off_dinv = o; o += (rp.Tri ? (size_t)rp.b * 8 : 0);
    o = (o + 15) & ~size_t(15);
    off_gth = o; o += (size_t)rp.sk_gd * TP * 8;
    size_t loop_bytes = o;
    size_t comb_bytes = off_stage + (size_t)tasks * CB * 8;
    off_red = 64;
    size_t epi_bytes = off_red + ((size_t)L + 2) * 8 + epilogue_doubles(rp) * 8;
    smem = std::max(std::max(loop_bytes, epi_bytes), comb_bytes);
    if (smem <= 220 * 1024 || T == 16) break;
    T /= 2;
  }
  const int limit = arith == 1 ? smem_limit<1>() : (arith == 2 ? smem_limit<2>() : smem_limit<0>());
  if ((long long)smem > limit) return RBO_ERR_ARG;
  const int ntiles = (int)((rp.n + T - 1) / T);
  const int occ = arith == 1 ? occupancy<1>((int)smem)
                             : (arith == 2 ? occupancy<2>((int)smem) : occupancy<0>((int)smem));
  int G = std::min(ntiles, occ * sm_count());
  if (rp.max_ctas > 0) G = std::min(G, rp.max_ctas);
  if (G < 1) G = 1;
  const int ngroups = (G + GROUP - 1) / GROUP;

  PassDev P;
  P.p = rp;
  P.T = T;
  P.TP = T + 2;
  P.ntiles = ntiles;
  P.items = items;
  P.cw = cw;
  P.nblk = nblk;
  for (int k = 0; k < 9; ++k) P.blk_start[k] = blk_start[k];
  P.tpo = tpo;
  P.tasks = tasks;
  // float-pair Gram chains are flushed into float64 after about 64 products
  P.flush_tiles = std::max(1, 64 / std::max(1, T / tpo));
  const bool alignedX = rp.a == 0 || (((uintptr_t)rp.X & 15) == 0 && (rp.ldx % 2) == 0);
  const bool alignedY = (((uintptr_t)rp.Y & 15) == 0 && (rp.ldy % 2) == 0);
  P.use_bulk = (alignedX && alignedY) ? 1 : 0;
  P.zr = zr;
  P.no = no;
  P.L = L;
  P.ngroups = ngroups;
  P.status = ar->status;
  P.off_stage = (int)off_stage;
  P.stage_bytes = (int)stage_bytes;
  P.off_c = (int)off_c;
  P.off_tri = (int)off_tri;
  P.off_dinv = (int)off_dinv;
  P.off_sk = 0;
  P.off_gth = (int)off_gth;
  P.rec_off = 0;
  P.off_ys = 0;
  P.ystage_bytes = 0;
  P.off_red = (int)off_red;
  P.partials = nullptr;
  P.gpart = nullptr;
  P.tickets = nullptr;
  if (L > 0) {
    // reduction scratch reserved for the whole call (stream-ordered reuse); the
    // tickets were zeroed at the start of the call and every tree resets its own
    const size_t need = ((size_t)G * L + (size_t)ngroups * L) * 8;
    if (ar->red == nullptr || need > ar->red_bytes) return RBO_ERR_NOMEM;
    if (ngroups + 1 > ar->n_tickets) return RBO_ERR_NOMEM;
    P.partials = ar->red;
    P.gpart = ar->red + (size_t)G * L;
    P.tickets = ar->tickets;
  }
  ProfToken tok = prof_start(st);
  if (arith == 1)
    rowpass_kernel<1><<<G, NT, smem, st>>>(P);
  else if (arith == 2)
    rowpass_kernel<2><<<G, NT, smem, st>>>(P);
  else
    rowpass_kernel<0><<<G, NT, smem, st>>>(P);
  if (prof_on()) {
    // algorithmic traffic: every n-row column read once, written once
    const double nn = (double)rp.n, A = rp.a, B = rp.b;
    const bool readx = rp.a > 0 && (rp.acc_x || rp.C);
    const double by = 8.0 * nn * ((readx ? A : 0.0) + B + (rp.write_y ? B : 0.0));
    double fl = 0.0;
    if (rp.C) fl += 2.0 * nn * A * B;                        // projection
    if (rp.Tri) fl += nn * B * B;                             // triangular solve
    if (rp.acc_x) fl += 2.0 * nn * A * B;                     // X^T Y'
    if (rp.acc_y) fl += nn * B * (B + 1.0);                   // Y'^T Y' (symmetric)
    if (rp.sk_d > 0) fl += nn * (double)rp.sk_zeta * B;       // sketch accumulation
    if (rp.sk_gd > 0) fl += 2.0 * nn * rp.sk_gd * B;          // Gaussian sketch
    prof_stop(tok, st, 0, by, fl, rp.tag);
  }
  if (launches) ++*launches;
  return note_cuda(cudaGetLastError());
}

// ------------------------------------------------------------------------------------
// sketch entries (tests / bit-exactness)
// ------------------------------------------------------------------------------------
__global__ void sketch_entries_kernel(int64_t row0, int64_t nrows, int d, int zeta, uint64_t seed,
                                      int32_t* idx, int8_t* sign, DevStatus* status) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int ix[ZMAX], ng[ZMAX];
#pragma unroll
  for (int t = 0; t < ZMAX; ++t) { ix[t] = 0; ng[t] = 0; }
  if (!sketch_column(seed, (uint64_t)(row0 + r), d, zeta, ix, ng)) set_error(status, RBO_ERR_SKETCH, 3);
#pragma unroll
  for (int t = 0; t < ZMAX; ++t) {
    if (t < zeta) {
      idx[r * zeta + t] = ix[t];
      sign[r * zeta + t] = ng[t] ? (int8_t)-1 : (int8_t)1;
    }
  }
}

// ------------------------------------------------------------------------------------
// sketch schedule (built once per call)
// ------------------------------------------------------------------------------------
int sketch_sched_mcap(int T, int d, int zeta) { return std::min(d, T * zeta); }

int sketch_sched_rec_bytes(int T, int d, int zeta) {
  return (sketch_sched_mcap(T, d, zeta) * 4 + T * zeta + 15) & ~15;
}

size_t sketch_sched_bytes(int64_t n, int T, int d, int zeta) {
  if (T <= 0 || n <= 0) return 0;
  return (size_t)((n + T - 1) / T) * (size_t)sketch_sched_rec_bytes(T, d, zeta);
}

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// ascending bitonic sort of N (a power of two) keys in shared memory, whole block
template <typename K>
__device__ void block_bitonic_sort(K* key, int N) {
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const K x = key[i], y = key[l];
          if ((x > y) == ((i & k) == 0)) {
            key[i] = y;
            key[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// One CTA per tile: hash the tile's rows (SplitMix64 sparse-sign columns), sort the
// (sketch row, pair) keys, then sort the non-empty sketch rows by entry count.
// Keys are unique, so the result does not depend on thread timing.
__global__ void sketch_sched_kernel(int64_t n, int T, int d, int zeta, uint64_t seed, int np2,
                                    int mp2, int mcap, int rec_bytes, uint8_t* out,
                                    DevStatus* status) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  unsigned long long* rkey = reinterpret_cast<unsigned long long*>(sm_raw);  // mp2
  uint32_t* key = reinterpret_cast<uint32_t*>(rkey + mp2);                    // np2
  __shared__ int s_nrow;
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int64_t r0 = (int64_t)tile * T;
  const int rows = (int)std::min<int64_t>((int64_t)T, n - r0);
  const int np = T * zeta;
  if (tid == 0) s_nrow = 0;
  for (int t = tid; t < np2; t += blockDim.x) key[t] = 0xFFFFFFFFu;
  for (int t = tid; t < mp2; t += blockDim.x) rkey[t] = ~0ull;
  __syncthreads();
  for (int r = tid; r < rows; r += blockDim.x) {
    int ix[ZMAX], ng[ZMAX];
#pragma unroll
    for (int t = 0; t < ZMAX; ++t) { ix[t] = 0; ng[t] = 0; }
    if (!sketch_column(seed, (uint64_t)(r0 + r), d, zeta, ix, ng)) set_error(status, RBO_ERR_SKETCH, 2);
#pragma unroll
    for (int t = 0; t < ZMAX; ++t) {
      if (t < zeta) {
        const uint32_t p = (uint32_t)(r * zeta + t);
        key[p] = ((uint32_t)ix[t] << 12) | (p << 1) | (uint32_t)ng[t];
      }
    }
  }
  __syncthreads();
  block_bitonic_sort(key, np2);
  uint8_t* rec = out + (size_t)tile * rec_bytes;
  uint32_t* meta = reinterpret_cast<uint32_t*>(rec);
  uint8_t* lst = rec + (size_t)mcap * 4;
  const int nvalid = rows * zeta;
  for (int q = tid; q < np; q += blockDim.x) {
    uint8_t v = 0;
    if (q < nvalid) {
      const uint32_t kq = key[q];
      const int p = (int)((kq >> 1) & 0x7FFu);
      v = (uint8_t)(((p / zeta) << 1) | (int)(kq & 1u));
      const uint32_t i = kq >> 12;
      if (q == 0 || (key[q - 1] >> 12) != i) {  // first entry of sketch row i
        int e = q + 1;
        while (e < nvalid && (key[e] >> 12) == i) ++e;
        const uint32_t cnt = (uint32_t)(e - q);
        const uint32_t m = i | ((uint32_t)q << 12) | (cnt << 23);
        const unsigned long long sk = ((unsigned long long)(511u - cnt) << 12) | i;
        const int slot = atomicAdd(&s_nrow, 1);
        rkey[slot] = (sk << 32) | m;
      }
    }
    lst[q] = v;
  }
  __syncthreads();
  block_bitonic_sort(rkey, mp2);
  for (int q = tid; q < mcap; q += blockDim.x)
    meta[q] = q < s_nrow ? (uint32_t)(rkey[q] & 0xFFFFFFFFull) : 0xFFFFFFFFu;
  // zero the record's padding
  for (int t = mcap * 4 + np + tid; t < rec_bytes; t += blockDim.x) rec[t] = 0;
}

int sketch_sched_launch(int64_t n, int T, int d, int zeta, uint64_t seed, uint8_t* out,
                        DevStatus* status, cudaStream_t st) {
  if (n <= 0 || (T != 16 && T != 32 && T != 64 && T != 128) || d < 1 || d > DMAX || zeta < 1 ||
      zeta > ZMAX || zeta > d || !out)
    return RBO_ERR_ARG;
  const int np2 = next_pow2(T * zeta), mcap = sketch_sched_mcap(T, d, zeta);
  const int mp2 = next_pow2(mcap);
  const size_t smem = (size_t)mp2 * 8 + (size_t)np2 * 4;
  const int64_t ntiles = (n + T - 1) / T;
  sketch_sched_kernel<<<(unsigned)ntiles, NT, smem, st>>>(n, T, d, zeta, seed, np2, mp2, mcap,
                                                          sketch_sched_rec_bytes(T, d, zeta), out,
                                                          status);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

int rowpass_sketch_T(int a_max, int b_max, int d, int zeta) {
  // shared memory of the streaming loop of a sketch pass (projection, no Gram); 128
  // rows only while a stage stays within STAGE_TARGET
  for (int T = 128; T > 16; T /= 2) {
    if (T > 64 && (size_t)(a_max + b_max) * (T + 2) * 8 > STAGE_TARGET) continue;
    if (rowpass_sk_loop_bytes(a_max, b_max, T, d, zeta) <= 220 * 1024) return T;
  }
  return 16;
}

int sketch_entries_launch(int64_t row0, int64_t nrows, int d, int zeta, uint64_t seed, int32_t* idx,
                          int8_t* sign, DevStatus* status, cudaStream_t st) {
  if (nrows <= 0) return RBO_OK;
  int64_t blocks = (nrows + 255) / 256;
  sketch_entries_kernel<<<(unsigned)blocks, 256, 0, st>>>(row0, nrows, d, zeta, seed, idx, sign, status);
  return cudaGetLastError() == cudaSuccess ? RBO_OK : RBO_ERR_CUDA;
}

}  // namespace rbo

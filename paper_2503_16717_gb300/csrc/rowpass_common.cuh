// Shared pieces of the row-pass kernels (rowpass.cu: float64 / float32 / float-pair
// arithmetic; ozaki.cu: tensor-core Gram with exact digit products): launch
// parameters, the small dense epilogue of the last CTA, and the fixed-order two-level
// tree that sums the per-CTA partials.
#pragma once

#include "device_common.cuh"
#include "small_dense.cuh"

namespace rbo {

constexpr int CB = 8;         // Z columns per task (register block)
constexpr int IPT = 4;        // Z tasks per thread
constexpr int GROUP = 16;     // CTAs per first-level reduction group
constexpr int NST = 2;        // pipeline stages
constexpr size_t STAGE_TARGET = 40 * 1024;  // bytes of one stage worth keeping in flight

struct PassDev {
  RowPass p;
  int T;              // rows per tile
  int TP;             // shared-memory column stride of a tile (T + 2: fewer bank conflicts)
  int ntiles;
  int items, tpo, tasks;  // Z work split: items = zr * (column blocks), tpo row subsets
  int cw;                 // width of every column block (<= CB)
  int nblk;               // column blocks
  int blk_start[9];       // first item of each block: X rows, then the Y' rows that reach
                          // the block (the symmetric Y'^T Y' needs no block below its diagonal)
  int flush_tiles;        // float-pair Gram: tiles between flushes into float64
  int use_bulk;       // X/Y aligned for 16-byte bulk copies
  int zr, no;         // Z rows, Z outputs (zr * b)
  int L;              // partial length (no + d*b)
  int ngroups;
  double* partials;
  double* gpart;
  unsigned* tickets;
  DevStatus* status;
  // shared memory layout (byte offsets from the dynamic base)
  int off_stage, stage_bytes, off_c, off_tri, off_dinv, off_sk, off_red;
  int off_gth;            // Gaussian sketch entries of the tile (sk_gd x TP)
  int rec_off;            // sketch schedule record of the tile, offset inside a stage
  int off_ys, ystage_bytes;  // sketch kernel: ring of Y stages (Y columns + record)
};

// ------------------------------------------------------------------------------------
// epilogue pieces
// ------------------------------------------------------------------------------------

// M = A * B for upper-triangular k x k matrices (ld k), all in global or shared memory.
static __device__ void tri_mult(const double* A, const double* B, int k, double* M) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e % k, c = e / k;
    double s = 0.0;
    for (int l = i; l <= c; ++l) s += A[i + l * k] * B[l + c * k];
    M[e] = (i <= c) ? s : 0.0;
  }
  __syncthreads();
}

// R assembly after the final Cholesky of a block (R2 in shared memory, k x k).
static __device__ void assemble(const Epilogue& e, const double* R2, int k, double* scratch,
                         DevStatus* status) {
  if (e.asm_op == ASM_NONE) return;
  double* Rf = e.Rfull;
  const int ld = e.ldR, p = e.p, c0 = e.col0;
  if (e.asm_op == ASM_DIAG) {
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
      int i = t % k, c = t / k;
      Rf[(p + i) + (size_t)(c0 + c) * ld] = R2[t];
    }
    __syncthreads();
    return;
  }
  // Loss of orthogonality: W~ = Qh - Q C2 is orthonormal up to O(eps kappa) terms
  // when the first intra-block step worked, so R2 = chol(W~^T W~) is close to I.
  // A large deviation means that step failed (the block is numerically rank
  // deficient at the working precision) and the final CholQR cannot repair it;
  // report instead of returning a non-orthogonal Q.
  if (threadIdx.x == 0) {
    double dev = 0.0;
    for (int t = 0; t < k * k; ++t) {
      const int i = t % k, c = t / k;
      if (i <= c) dev = fmax(dev, fabs(R2[t] - (i == c ? 1.0 : 0.0)));
    }
    if (!(dev <= 0.5)) {
      if (atomicCAS(&status->code, 0, RBO_ERR_LOST_ORTHOGONALITY) == 0) {
        status->block = e.block;
        status->column = -1;
        status->stage = RBO_STAGE_FINAL;
      }
    }
  }
  // M = R' * (R_hat or T)
  double* M = scratch;  // k x k
  tri_mult(e.Rp, e.Rh, k, M);
  // R_jj = R2 M
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int i = t % k, c = t / k;
    double s = 0.0;
    for (int l = i; l <= c; ++l) s += R2[i + l * k] * M[l + c * k];
    Rf[(p + i) + (size_t)(c0 + c) * ld] = (i <= c) ? s : 0.0;
  }
  // R_top = C1 + C2 M
  for (int t = threadIdx.x; t < p * k; t += blockDim.x) {
    int i = t % p, c = t / p;
    double s = e.C1[i + (size_t)c * e.ldc1];
    for (int l = 0; l <= c; ++l) s += e.C2[i + (size_t)l * e.ldc2] * M[l + c * k];
    Rf[i + (size_t)(c0 + c) * ld] = s;
  }
  if (e.asm_op == ASM_TWO_STAGE && e.coords != nullptr) {
    // coordinates of Qbar_B in [Q, Q_B]: [C2 R'; R2 R']
    for (int t = threadIdx.x; t < (p + k) * k; t += blockDim.x) {
      int i = t % (p + k), c = t / (p + k);
      double s = 0.0;
      if (i < p) {
        for (int l = 0; l <= c; ++l) s += e.C2[i + (size_t)l * e.ldc2] * e.Rp[l + c * k];
      } else {
        int ii = i - p;
        for (int l = ii; l <= c; ++l) s += R2[ii + l * k] * e.Rp[l + c * k];
      }
      e.coords[i + (size_t)c * e.ldcoords] = s;
    }
  }
  __syncthreads();
}

// Rows of the sketch S Y' a pass produces (after the Count-Gauss Gaussian stage).
__host__ __device__ inline int sketch_rows(const RowPass& rp) {
  return rp.sk_gd > 0 ? rp.sk_gd : (rp.sk_cg > 0 ? rp.sk_cg : rp.sk_d);
}

// The reduced sketch S Y' (sketch_rows x b, column-major) into A: sparse-sign from
// the scattered part of the partial; Gaussian from its Z rows; Count-Gauss as G times
// the scattered Count stage, G generated here (float32 Box-Muller, as in the tiles).
static __device__ void load_sketch(const PassDev& P, const double* red, double* A) {
  const RowPass& rp = P.p;
  const int b = rp.b, d = sketch_rows(rp);
  if (rp.sk_gd > 0) {
    for (int t = threadIdx.x; t < d * b; t += blockDim.x) A[t] = red[(t % d) * b + t / d];
  } else if (rp.sk_cg > 0) {
    const int di = rp.sk_d;
    for (int t = threadIdx.x; t < d * b; t += blockDim.x) {
      const int k = t % d, c = t / d;
      double s = 0.0;
      for (int j = 0; j < di; ++j)
        s = fma((double)gauss_entry(rp.sk_seed, (uint64_t)j, k, d), red[P.no + j + (size_t)c * di], s);
      A[t] = s;
    }
  } else {
    for (int t = threadIdx.x; t < d * b; t += blockDim.x) A[t] = red[P.no + t];
  }
  __syncthreads();
}

// The small dense work of the last CTA.  `red` holds the reduced partial
// (Z: zr x b as o = i*b + c, then the scattered sketch d x b column-major); `sm` is
// free shared memory.
static __device__ void run_epilogue(const PassDev& P, const double* red, double* sm, int* s_flag) {
  const RowPass& rp = P.p;
  const Epilogue& e = rp.epi;
  const int b = rp.b;
  const int ax = rp.sk_gd + (rp.acc_x ? rp.a : 0);
  switch (e.op) {
    case EPI_STORE: {
      for (int t = threadIdx.x; t < ax * b; t += blockDim.x) {
        int i = t / b, c = t % b;
        e.out[(e.row_off + i) + (size_t)(e.col_off + c) * e.out_ld] = red[t];
      }
      break;
    }
    case EPI_STORE_ALL: {
      for (int t = threadIdx.x; t < P.zr * b; t += blockDim.x) {
        int i = t / b, c = t % b;
        e.out[i + (size_t)c * P.zr] = red[t];
      }
      if (e.out_sk != nullptr)
        for (int t = threadIdx.x; t < rp.sk_d * b; t += blockDim.x) e.out_sk[t] = red[P.no + t];
      break;
    }
    case EPI_CHOL: {
      double* G = sm;  // b x b
      for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
        int i = t % b, c = t / b;
        G[t] = red[(ax + i) * b + c];
      }
      __syncthreads();
      int bad = cta_cholesky(G, b, s_flag);
      if (bad >= 0) {
        if (threadIdx.x == 0) set_breakdown(P.status, e.block, bad, e.stage);
        return;
      }
      if (e.out_r != nullptr)
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) e.out_r[t] = G[t];
      __syncthreads();
      assemble(e, G, b, sm + b * b, P.status);
      break;
    }
    case EPI_PIP: {
      // Pythagorean rule (Section 7.1): the Gram of Vh - Qbar P is G - P^T P
      const int pp = ax, k = b, K = e.K, off = e.poff;
      double* S = sm;  // k x k
      for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int i = t % k, c = t / k;
        double v = red[(pp + i) * b + c];
        for (int l = 0; l < pp; ++l) v -= red[l * b + i] * red[l * b + c];
        S[t] = v;
      }
      __syncthreads();
      const int bad = cta_cholesky(S, k, s_flag);
      if (bad >= 0) {
        if (threadIdx.x == 0) set_breakdown(P.status, e.block, off + bad, e.stage);
        return;
      }
      for (int t = threadIdx.x; t < pp * k; t += blockDim.x) {
        const int l = t % pp, c = t / pp;
        e.T[l + (size_t)(off + c) * K] = red[l * b + c];
      }
      for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int i = t % k, c = t / k;
        e.T[(off + i) + (size_t)(off + c) * K] = (i <= c) ? S[t] : 0.0;
      }
      break;
    }
    case EPI_SKETCH_OUT: {
      load_sketch(P, red, sm);
      for (int t = threadIdx.x; t < sketch_rows(rp) * b; t += blockDim.x) e.out_sk[t] = sm[t];
      break;
    }
    case EPI_HH: {
      const int d = sketch_rows(rp);
      double* A = sm;                      // d x b
      double* R = A + (size_t)d * b;       // b x b
      double* beta = R + b * b;            // b
      double* sg = beta + b;               // b
      double* scr = sg + b;                // 32
      load_sketch(P, red, A);
      cta_householder(A, d, b, R, nullptr, beta, sg, scr);
      __syncthreads();
      if (threadIdx.x == 0) {
        const int bad = tri_rank_deficient(R, b);
        if (bad >= 0) set_breakdown(P.status, e.block, bad, e.stage);
      }
      for (int t = threadIdx.x; t < b * b; t += blockDim.x) e.out_r[t] = R[t];
      break;
    }
    case EPI_SKB2: {
      // sketched BCGS2 with Householder intra step (Section 7.2)
      const int d = sketch_rows(rp), k = b, pp = e.poff, K = e.K;
      double* v = sm;                       // d x k
      double* A = v + (size_t)d * k;        // d x k (Householder work)
      double* Qn = A + (size_t)d * k;       // d x k
      double* c1 = Qn + (size_t)d * k;      // pp x k
      double* c2 = c1 + (size_t)pp * k;     // pp x k
      double* R = c2 + (size_t)pp * k;      // k x k
      double* beta = R + k * k;
      double* sg = beta + k;
      double* scr = sg + k;
      if (pp > 0) cta_prefetch_cols(e.qs, d, d, pp);
      load_sketch(P, red, v);
      if (pp > 0) {
        cta_gemm_tn(e.qs, d, v, d, pp, k, c1);
        cta_gemm_nn_sub(e.qs, d, c1, d, pp, k, v);
        cta_gemm_tn(e.qs, d, v, d, pp, k, c2);
        cta_gemm_nn_sub(e.qs, d, c2, d, pp, k, v);
        for (int t = threadIdx.x; t < pp * k; t += blockDim.x) {
          int i = t % pp, c = t / pp;
          e.T[i + (size_t)(pp + c) * K] = c1[t] + c2[t];
        }
      }
      for (int t = threadIdx.x; t < d * k; t += blockDim.x) A[t] = v[t];
      __syncthreads();
      cta_householder(A, d, k, R, Qn, beta, sg, scr);
      __syncthreads();
      if (threadIdx.x == 0) {
        const int bad = tri_rank_deficient(R, k);
        if (bad >= 0) set_breakdown(P.status, e.block, pp + bad, e.stage);
      }
      for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        int i = t % k, c = t / k;
        e.T[(pp + i) + (size_t)(pp + c) * K] = R[t];
      }
      for (int t = threadIdx.x; t < d * k; t += blockDim.x) {
        int r = t % d, c = t / d;
        e.qs[r + (size_t)(pp + c) * d] = Qn[t];
      }
      break;
    }
    case EPI_GB: {
      // block column [Qbar_prev, Qbar_j]^T Qbar_j of the big-panel Gram G_B
      const int K = e.K, pp = e.poff;
      for (int t = threadIdx.x; t < P.zr * b; t += blockDim.x) {
        int i = t / b, c = t % b;
        e.GB[i + (size_t)(pp + c) * K] = red[t];
      }
      __threadfence_block();
      __syncthreads();
      if (e.last) {
        const int Kc = pp + b;  // columns of the big panel
        double* G = sm;
        for (int t = threadIdx.x; t < Kc * Kc; t += blockDim.x) {
          int i = t % Kc, c = t / Kc;
          G[t] = (i <= c) ? e.GB[i + (size_t)c * K] : 0.0;
        }
        __syncthreads();
        int bad = cta_cholesky(G, Kc, s_flag);
        if (bad >= 0) {
          if (threadIdx.x == 0) set_breakdown(P.status, e.block, bad, RBO_STAGE_BIGPANEL);
          return;
        }
        for (int t = threadIdx.x; t < Kc * Kc; t += blockDim.x) e.out_rp[t] = G[t];
      }
      break;
    }
    default:
      break;
  }
  __syncthreads();
}


// Fixed-order two-level tree over the per-CTA partials (each CTA has written its L
// values to P.partials + blockIdx.x * L): groups of GROUP CTAs are summed by the
// group's last CTA (ticket), then the last group summer sums the group partials into
// shared memory and runs the small dense epilogue.  Every sum has a fixed order, so
// the result is bitwise reproducible.  `smem` is the kernel's dynamic shared memory.
__device__ __forceinline__ void tree_reduce_epilogue(const PassDev& P, unsigned char* smem,
                                                     int* s_flag, int* s_last_p) {
  const int tid = threadIdx.x;
  int& s_last = *s_last_p;
  __threadfence();
  __syncthreads();
  const int g = blockIdx.x / GROUP;
  const int gsize = min(GROUP, (int)gridDim.x - g * GROUP);
  if (tid == 0) {
    unsigned prev = atomicAdd(&P.tickets[g], 1u);
    s_last = (prev == (unsigned)(gsize - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  {
    const double* base = P.partials + (size_t)g * GROUP * P.L;
    double* gout = P.gpart + (size_t)g * P.L;
    for (int t = tid; t < P.L; t += (int)blockDim.x) {
      double s = 0.0;
      double v[GROUP];
#pragma unroll
      for (int i = 0; i < GROUP; ++i) v[i] = i < gsize ? __ldcg(base + (size_t)i * P.L + t) : 0.0;
#pragma unroll
      for (int i = 0; i < GROUP; ++i)
        if (i < gsize) s += v[i];
      gout[t] = s;
    }
  }
  if (tid == 0) P.tickets[g] = 0u;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned prev = atomicAdd(&P.tickets[P.ngroups], 1u);
    s_last = (prev == (unsigned)(P.ngroups - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double* red = reinterpret_cast<double*>(smem + P.off_red);
  for (int t = tid; t < P.L; t += (int)blockDim.x) {
    double s = 0.0;
    for (int i0 = 0; i0 < P.ngroups; i0 += 8) {
      double v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        v[i] = i0 + i < P.ngroups ? __ldcg(P.gpart + (size_t)(i0 + i) * P.L + t) : 0.0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (i0 + i < P.ngroups) s += v[i];
    }
    red[t] = s;
  }
  if (tid == 0) P.tickets[P.ngroups] = 0u;
  __syncthreads();
  double* sm = red + ((P.L + 1) & ~1);
  run_epilogue(P, red, sm, s_flag);
}

// shared memory bytes of the small dense epilogue (beyond the reduced vector)
static inline size_t epilogue_doubles(const RowPass& rp) {
  const int b = rp.b, d = sketch_rows(rp);
  const Epilogue& e = rp.epi;
  size_t need = 0;
  switch (e.op) {
    case EPI_CHOL: need = (size_t)b * b * 2 + 64; break;
    case EPI_HH: need = (size_t)d * b + (size_t)b * b + 2 * b + 64; break;
    case EPI_SKB2: need = (size_t)3 * d * b + (size_t)2 * e.poff * b + (size_t)b * b + 2 * b + 64; break;
    case EPI_GB: need = (size_t)(e.poff + b) * (e.poff + b) + 64; break;
    case EPI_PIP: need = (size_t)b * b + 64; break;
    case EPI_SKETCH_OUT: need = (size_t)d * b + 64; break;
    default: break;
  }
  return need;
}

// ------------------------------------------------------------------------------------
// sketch entry sums of one tile (both row-pass kernels)
// ------------------------------------------------------------------------------------
// Sketch of one sketch row over a tile, float64 path: the tile's values of each column
// are held as int64 fixed point (unit 2^(E_c - 1077), E_c the column's largest
// exponent field in the tile; fix_from_double); the row's entries are summed exactly
// in integers (signs by integer negation), and the exact tile sum is rounded once to
// float64 and added to the accumulator: one float64 add per (sketch row, column) and
// tile instead of one per entry, on every lane.  A column with a non-finite value in
// the tile (E_c = 0x7FF) makes the accumulators NaN.
template <int CW>
__device__ __forceinline__ void sketch_row_fix(double* acc, int d, const long long* y, int TP,
                                               const int* emax, const uint8_t* e, int cnt) {
  long long v[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) v[c] = 0;
  for (int t = 0; t < cnt; ++t) {
    const int ev = e[t];
    const int r = ev >> 1;
    const long long ng = -(long long)(ev & 1);  // 0 or all ones
#pragma unroll
    for (int c = 0; c < CW; ++c) {
      const long long f = y[(size_t)c * TP + r];
      v[c] += (f ^ ng) - ng;                     // f or -f
    }
  }
#pragma unroll
  for (int c = 0; c < CW; ++c) {
    const double add = emax[c] == 0x7FF ? __longlong_as_double(0x7FF8000000000000LL)
                                        : double_from_fix(v[c], emax[c]);
    acc[(size_t)c * d] += add;
  }
}
// float32 values in the first 4 bytes of each 8-byte slot: y holds 2 floats per row
template <int CW>
__device__ __forceinline__ void sketch_row_f32(float* acc, int d, const float* y, int TP2,
                                               const uint8_t* e, int cnt) {
  float v[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) v[c] = acc[(size_t)c * d];
  for (int t = 0; t < cnt; ++t) {
    const int ev = e[t];
    const int r = 2 * (ev >> 1);
    const int sg = (ev & 1) << 31;
#pragma unroll
    for (int c = 0; c < CW; ++c) v[c] += __int_as_float(__float_as_int(y[(size_t)c * TP2 + r]) ^ sg);
  }
#pragma unroll
  for (int c = 0; c < CW; ++c) acc[(size_t)c * d] = v[c];
}
#define RBO_CW_DISPATCH(fn, cw, ...)            \
  switch (cw) {                                 \
    case 8: fn<8>(__VA_ARGS__); break;          \
    case 7: fn<7>(__VA_ARGS__); break;          \
    case 6: fn<6>(__VA_ARGS__); break;          \
    case 5: fn<5>(__VA_ARGS__); break;          \
    case 4: fn<4>(__VA_ARGS__); break;          \
    case 3: fn<3>(__VA_ARGS__); break;          \
    case 2: fn<2>(__VA_ARGS__); break;          \
    default: fn<1>(__VA_ARGS__); break;         \
  }

}  // namespace rbo

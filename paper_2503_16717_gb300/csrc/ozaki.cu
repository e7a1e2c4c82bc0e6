// Tensor-core Gram pass: Z = [X Y']^T Y' with float64 accuracy from exact products of
// 8-bit digits on the bf16 tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// The Gram matrices of BCGS and CholQR (Sections 4-5, the reductions Q^T W and W^T W)
// are the float64 contractions of the method.  On this GPU the float64 pipe (2 FMA per
// SM per clock) caps a float64 Gram pass near 1.1 TFLOP/s, far below the HBM rate, while
// the bf16 tensor cores are three orders of magnitude faster.  Splitting every float64
// value into digits that bf16 represents exactly turns the Gram into exact integer
// products (the idea of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012):
//
//   * per tile of T = 128 rows and per column c, E_c = the largest exponent field of
//     the column in the tile; every value becomes the integer F = x 2^(1076 - E_c)
//     rounded to nearest, |F| < 2^54 (an error of at most 2^-54 of the column's
//     largest magnitude in the tile);
//   * G = F + 0x0080808080808080 lies in [0, 2^56) (the balanced range of 7 bytes is
//     +-0x7F7F7F7F7F7F7F > 2^54); byte k of G minus 128 is the balanced digit d_k in
//     [-128, 127] and F = sum_k d_k 2^(8k) exactly; digit I = 0..6 is byte 6 - I (most
//     significant first), each exact in bf16;
//   * one tensor-core product of a digit of x and a digit of y is an integer of at most
//     2^14 in magnitude, so a sum over the 128 rows of a tile is an integer below 2^21,
//     exact in the float32 accumulator whatever the order of the additions;
//   * the digit pairs (I, J) with I + J <= 7 are kept (the dropped ones weigh less than
//     2^-57 of the product of the two columns' largest magnitudes); per tile they are
//     combined in 64-bit integers and added, shifted by the tile's exponents, into a
//     128-bit integer accumulator per output; the per-CTA value is rounded to float64
//     once.
//
// Tensor-core mapping (M = 128, K = 16 rows per instruction):
//   A (tensor memory): lane (p, c) = column c of [X Y'] (c < 64) with digits of parity p:
//     region q = 0..3 of a K-step holds digit I = 2q + p (zero for I = 7);
//   B (shared memory, no-swizzle K-major): row 8 yc + J = digit J of column yc of Y';
//   D_q (tensor memory, one region per q): D_q[(p, c), 8 yc + J] = sum over the tile's
//     rows of digit (2q + p) of x_c times digit J of y'_yc.
// Per K-step 4 instructions; the regions are independent accumulators.
//
// Supported passes: Gram of [X Y']^T Y' (acc_x and/or acc_y) with a + b <= 64 columns in
// A, b <= 8, optionally after the triangular solve y' = y Tri^-1 (float64, written
// back).  Everything after the per-CTA partials (the fixed-order tree and the small
// dense epilogue) is shared with the float64 row pass.
#include <algorithm>
#include <mutex>

#include "rowpass_common.cuh"

namespace rbo {
namespace {

constexpr int OZ_T = 128;            // rows per tile (the exponent chunk)
constexpr int OZ_KS = OZ_T / 16;     // tensor-core K-steps per tile
constexpr int OZ_NT = 256;           // two warpgroups
constexpr int OZ_MAXA = 64;          // columns of [X Y'] in A
constexpr int OZ_MAXB = 8;           // columns of Y'
constexpr uint32_t OZ_TMEM_COLS = 512;
constexpr unsigned long long OZ_BIAS = 0x0080808080808080ULL;
static_assert(OZ_NT == NT, "the shared tree reduction strides by NT");

struct OzDev {
  PassDev P;
  int nA;      // columns of A: a (acc_x) then b (acc_y)
  int N;       // MMA N = 16 ceil(8 b / 16)
  int off_B;   // B digit tiles: OZ_KS x N rows x 32 bytes
};

// ---- PTX: tensor memory and the tensor-core MMA (tcgen05) ------------------------------
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // no-swizzle canonical layout: start >> 4, leading (K) byte offset >> 4, stride (M/N)
  // byte offset >> 4, descriptor version 1 (bits 46-48 = 0b001)
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}
// kind::f16 instruction descriptor: D float32, A and B bf16, both K-major, N >> 3, M >> 4
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
      "%29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
      "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
      "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
// 32 columns of this warp's lane quarter; the wait is in the same statement, so the
// registers are complete when the statement ends
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];\n\ttcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- digits -----------------------------------------------------------------------------
// Digit I (0 = most significant) of the biased fixed point G as a float (an integer in
// [-128, 127]): byte 6 - I of G placed in the low byte of 2^23 (0x4B000000), minus
// 2^23 + 128.
__device__ __forceinline__ float digit_f(uint32_t glo, uint32_t ghi, int I) {
  const int k = 6 - I;
  const uint32_t w = k >= 4 ? ghi : glo;
  return __int_as_float((int)__byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)(k & 3))) - 8388736.0f;
}
// bf16 pair (x: low half, y: high half) of two floats that bf16 represents exactly
__device__ __forceinline__ uint32_t pack_bf16(float x, float y) {
  return __byte_perm(__float_as_uint(x), __float_as_uint(y), 0x7632u);
}
// F = y 2^(1076 - E) rounded to nearest (ties away from zero), |F| < 2^54 for a value
// whose exponent field is at most E; zero and subnormal values give 0
__device__ __forceinline__ long long oz_fix(double y, int E) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(y);
  const int e = (int)((u >> 52) & 0x7FF);
  if (e == 0) return 0;
  const unsigned long long M = (u & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const int sh = e - E + 1;  // <= 1
  unsigned long long v;
  if (sh >= 0) {
    v = M << sh;
  } else if (sh > -64) {
    const int k = -sh;
    v = (M + (1ULL << (k - 1))) >> k;
  } else {
    v = 0;
  }
  return (u >> 63) ? -(long long)v : (long long)v;
}
__device__ __forceinline__ void biased_fix(double v, int E, uint32_t& lo, uint32_t& hi) {
  const unsigned long long g = (unsigned long long)oz_fix(v, E) + OZ_BIAS;
  lo = (uint32_t)g;
  hi = (uint32_t)(g >> 32);
}
// an exact integer-valued float of magnitude below 2^22 to int
__device__ __forceinline__ int f2i_exact(float v) {
  return __float_as_int(v + 12582912.0f) - 0x4B400000;
}

// ---- the kernel ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OZ_NT, 1) ozaki_gram_kernel(const __grid_constant__ OzDev D) {
  const PassDev& P = D.P;
  const RowPass& rp = P.p;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_flag;
  __shared__ int s_last;
  __shared__ uint32_t s_tmem;
  __shared__ int s_E[OZ_MAXA + OZ_MAXB];    // exponent field maximum per column, this tile
  __shared__ int s_bad[OZ_MAXA + OZ_MAXB];  // a non-finite value met in the column
  __shared__ __align__(8) uint64_t s_mma_bar;
  if (read_code(P.status) != 0) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, wg = warp >> 2;
  const int a = rp.a, b = rp.b, T = OZ_T, TP = P.TP;
  const int ncol = a + b;     // staged columns: X then Y
  const int nA = D.nA, N = D.N;
  const int64_t n = rp.n;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  double* Ts = reinterpret_cast<double*>(smem + P.off_tri);
  double* dinv = reinterpret_cast<double*>(smem + P.off_dinv);
  unsigned char* Bs = smem + D.off_B;

  if (rp.Tri) {
    const int ldt = rp.ldtri > 0 ? rp.ldtri : b;
    for (int t = tid; t < b * b; t += OZ_NT) {
      const int i = t % b, c = t / b;
      Ts[t] = (i <= c) ? rp.Tri[i + (size_t)c * ldt] : 0.0;
    }
    for (int t = tid; t < b; t += OZ_NT) dinv[t] = 1.0 / rp.Tri[t + (size_t)t * ldt];
  }
  // B tiles: rows 8 yc + 7 and rows >= 8 b stay zero
  for (int t = tid; t < OZ_KS * N * 8; t += OZ_NT) reinterpret_cast<uint32_t*>(Bs)[t] = 0u;
  for (int t = tid; t < OZ_MAXA + OZ_MAXB; t += OZ_NT) s_bad[t] = 0;
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
    mbar_init(&s_mma_bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tA = s_tmem;          // A: K-step ks, region q at columns 32 ks + 8 q
  const uint32_t tD = s_tmem + 256;    // D_q at columns 256 + q N
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  // this thread's A lane: (parity p, column c)
  const int L = 32 * (warp & 3) + lane;
  const int par = L >> 6, xc = L & 63;
  const bool active = xc < nA;

  // 128-bit integer accumulators: value = acc[yc] * 2^(ea[yc] - 2112)
  __int128 acc[OZ_MAXB];
  int ea[OZ_MAXB];
#pragma unroll
  for (int c = 0; c < OZ_MAXB; ++c) {
    acc[c] = 0;
    ea[c] = -1;
  }

  auto stage_X = [&](int s) {
    return reinterpret_cast<double*>(smem + P.off_stage + (size_t)s * P.stage_bytes);
  };
  auto issue_tile = [&](int tile, int s) {
    const int64_t r0 = (int64_t)tile * T;
    double* xs = stage_X(s);
    const uint32_t bytes = (uint32_t)T * 8u;
    if (lane == 0) mbar_arrive_expect_tx(&bars[s], bytes * (uint32_t)ncol);
    __syncwarp();
    for (int j = lane; j < ncol; j += 32) {
      const double* src = j < a ? rp.X + j * rp.ldx + r0 : rp.Y + (j - a) * rp.ldy + r0;
      bulk_copy_g2s(xs + (size_t)j * TP, src, bytes, &bars[s]);
    }
  };
  auto bulk_ok = [&](int tile) { return P.use_bulk && ((int64_t)(tile + 1) * T <= n); };

  uint32_t phase[NST] = {0u, 0u};
  uint32_t mma_phase = 0u;
  bool failed = false;
  const int first = blockIdx.x;
  if (first < P.ntiles && bulk_ok(first) && warp == 0) issue_tile(first, 0);

  int it = 0;
  for (int tile = first; tile < P.ntiles; tile += gridDim.x, ++it) {
    const int s = it & 1;
    const int64_t r0 = (int64_t)tile * T;
    const int rows = (n - r0 < (int64_t)T) ? (int)(n - r0) : T;
    double* xs = stage_X(s);
    double* ys = xs + (size_t)a * TP;
    if (bulk_ok(tile)) {
      const bool ok = mbar_wait_bounded(&bars[s], phase[s]);
      phase[s] ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) set_error(P.status, RBO_ERR_TIMEOUT, 11);
        failed = true;
        break;
      }
    } else {
      for (int t = tid; t < ncol * T; t += OZ_NT) {
        const int col = t / T, r = t % T;
        double v = 0.0;
        if (r < rows) v = (col < a) ? rp.X[col * rp.ldx + r0 + r] : rp.Y[(col - a) * rp.ldy + r0 + r];
        xs[(size_t)col * TP + r] = v;
      }
      __syncthreads();
    }
    const int nxt = tile + gridDim.x;
    if (warp == 0 && nxt < P.ntiles && bulk_ok(nxt)) {
      fence_proxy_async();
      issue_tile(nxt, s ^ 1);
    }

    // ---- y' = y Tri^-1 (float64), written back --------------------------------------
    if (rp.Tri) {
      for (int c0 = 0; c0 < b; c0 += CB) {
        const int cw = min(CB, b - c0);
        if (c0 > 0) {
          for (int t = tid; t < T * cw; t += OZ_NT) {
            const int r = t % T, c = c0 + t / T;
            double v = ys[c * TP + r];
            for (int i = 0; i < c0; ++i) v = fma(-ys[i * TP + r], Ts[i + c * b], v);
            ys[c * TP + r] = v;
          }
          __syncthreads();
        }
        for (int r = tid; r < T; r += OZ_NT) {
          for (int c = c0; c < c0 + cw; ++c) {
            double v = ys[c * TP + r];
            for (int i = c0; i < c; ++i) v = fma(-ys[i * TP + r], Ts[i + c * b], v);
            ys[c * TP + r] = v * dinv[c];
          }
        }
        __syncthreads();
      }
      if (rp.write_y)
        for (int t = tid; t < b * T; t += OZ_NT) {
          const int c = t / T, rr = t % T;
          if (rr < rows) rp.Y[c * rp.ldy + r0 + rr] = ys[(size_t)c * TP + rr];
        }
    }

    // ---- exponent field maxima of the tile's columns ----------------------------------
    for (int c = tid; c < ncol; c += OZ_NT) s_E[c] = 0;
    __syncthreads();
    for (int t = tid; t < ncol * T; t += OZ_NT) {
      const int c = t / T, r = t % T;   // T a multiple of 32: a warp shares one column
      const uint32_t hi = (uint32_t)__double2hiint(xs[(size_t)c * TP + r]);
      int ex = (int)((hi >> 20) & 0x7FFu);
      ex = __reduce_max_sync(0xffffffffu, ex);
      if (lane == 0 && ex != 0) atomicMax(&s_E[c], ex);
    }
    __syncthreads();
    for (int c = tid; c < ncol; c += OZ_NT)
      if (s_E[c] == 0x7FF) s_bad[c] = 1;

    // ---- digits: A into tensor memory, B into shared memory ----------------------------
    for (int ks = wg; ks < OZ_KS; ks += 2) {
      uint32_t w[32];
      if (active) {
        const double* col = xs + (size_t)xc * TP + ks * 16;
        const int E = s_E[xc];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const double2 v = *reinterpret_cast<const double2*>(col + 2 * j);
          uint32_t g0l, g0h, g1l, g1h;
          biased_fix(v.x, E, g0l, g0h);
          biased_fix(v.y, E, g1l, g1h);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int I = 2 * q + par;
            w[q * 8 + j] = I <= 6 ? pack_bf16(digit_f(g0l, g0h, I), digit_f(g1l, g1h, I)) : 0u;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) w[j] = 0u;
      }
      tmem_st32(tA + (uint32_t)(32 * ks) + lane_base, w);
      // B: Y' digits of the K-step's 16 rows, row 8 yc + J of the K-major tile
      unsigned char* Bk = Bs + (size_t)ks * N * 32;
      for (int e = tid & 127; e < 16 * b; e += 128) {
        const int r = e & 15, yc = e >> 4;
        uint32_t gl, gh;
        biased_fix(ys[(size_t)yc * TP + ks * 16 + r], s_E[a + yc], gl, gh);
#pragma unroll
        for (int J = 0; J < 7; ++J) {
          const int nrow = 8 * yc + J;
          const uint32_t bits = __float_as_uint(digit_f(gl, gh, J)) >> 16;
          *reinterpret_cast<uint16_t*>(Bk + (nrow >> 3) * 256 + (r >> 3) * 128 + (nrow & 7) * 16 +
                                       (r & 7) * 2) = (uint16_t)bits;
        }
      }
    }
    tmem_wait_st();
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();

    // ---- tensor-core products of the tile ------------------------------------------------
    if (tid == 0) {
      tc_fence_after();
      const uint32_t id = idesc_bf16(128, N);
      for (int ks = 0; ks < OZ_KS; ++ks) {
        const uint64_t db = smem_desc(smem_u32(Bs + (size_t)ks * N * 32), 128, 256);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          mma_ts(tD + (uint32_t)(q * N), tA + (uint32_t)(32 * ks + 8 * q), db, id, ks > 0 ? 1u : 0u);
      }
      mma_commit(&s_mma_bar);
    }
    __syncwarp();
    const bool done = mbar_wait_bounded(&s_mma_bar, mma_phase);
    mma_phase ^= 1u;
    tc_fence_after();
    if (__syncthreads_or(!done)) {
      if (tid == 0) set_error(P.status, RBO_ERR_TIMEOUT, 12);
      mbar_wait_bounded(&s_mma_bar, mma_phase ^ 1u);  // a second bounded chance before freeing
      failed = true;
      break;
    }

    // ---- drain: warpgroup wg reads the regions q = 2 wg, 2 wg + 1 ------------------------
    {
      long long hi[OZ_MAXB], lo[OZ_MAXB];
#pragma unroll
      for (int c = 0; c < OZ_MAXB; ++c) { hi[c] = 0; lo[c] = 0; }
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int q = 2 * wg + qq;
        const int I = 2 * q + par;
        float v[64];
        tmem_ld32(tD + (uint32_t)(q * N) + lane_base, v);
        tmem_ld32(tD + (uint32_t)(q * N + 32) + lane_base, v + 32);
        if (active && I <= 6) {
#pragma unroll
          for (int yc = 0; yc < OZ_MAXB; ++yc) {
            if (yc < b) {
#pragma unroll
              for (int J = 0; J < 7; ++J) {
                const int Lv = I + J;
                if (Lv <= 7) {
                  const long long iv = (long long)f2i_exact(v[8 * yc + J]);
                  if (Lv <= 3) hi[yc] += iv << (8 * (3 - Lv));
                  else lo[yc] += iv << (8 * (7 - Lv));
                }
              }
            }
          }
        }
      }
      if (active) {
#pragma unroll
        for (int yc = 0; yc < OZ_MAXB; ++yc) {
          if (yc < b) {
            const __int128 S = ((__int128)hi[yc] << 32) + (__int128)lo[yc];
            if (S != 0) {
              const int Tt = s_E[xc] + s_E[a + yc];
              if (ea[yc] < 0) ea[yc] = Tt;
              int sh = Tt - ea[yc];
              // |S| < 2^80; a shift of at most 24 keeps the sum of the CTA's tiles far
              // below 2^127
              if (sh > 24) {  // magnitude grew: renormalise the accumulator
                acc[yc] >>= (sh - 24);
                ea[yc] += sh - 24;
                sh = 24;
              }
              if (sh >= 0) acc[yc] += S << sh;
              else if (sh > -120) acc[yc] += S >> (-sh);
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // D, A, B and stage s free for the next tile
  }

  // ---- free the tensor memory ---------------------------------------------------------------
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem),
                 "r"(OZ_TMEM_COLS));
  }
  if (failed || P.L == 0) return;

  // ---- per-CTA partial: four threads hold parts of every output ----------------------------
  double* comb = reinterpret_cast<double*>(smem + P.off_stage);  // 4 x 64 x 8
#pragma unroll
  for (int yc = 0; yc < OZ_MAXB; ++yc) {
    double v = 0.0;
    if (ea[yc] >= 0) v = ldexp((double)acc[yc], ea[yc] - 2112);
    comb[((size_t)(wg * 2 + par) * OZ_MAXA + xc) * OZ_MAXB + yc] = v;
  }
  __syncthreads();
  double* mypart = P.partials + (size_t)blockIdx.x * P.L;
  for (int o = tid; o < P.no; o += OZ_NT) {
    const int i = o / b, c = o % b;
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) sum += comb[((size_t)k * OZ_MAXA + i) * OZ_MAXB + c];
    if (s_bad[i] || s_bad[a + c]) sum = __longlong_as_double(0x7FF8000000000000LL);
    mypart[o] = sum;
  }
  tree_reduce_epilogue(P, smem, &s_flag, &s_last);
}

std::mutex g_oz_mu;
int g_oz_smem_set[64] = {};

}  // namespace

bool ozaki_gram_supported(const RowPass& rp) {
  if (!rp.ozaki || rp.C || rp.sk_d > 0 || rp.sk_gd > 0 || rp.mixed || rp.df64) return false;
  if (!rp.acc_x && !rp.acc_y) return false;
  if (rp.b < 1 || rp.b > OZ_MAXB) return false;
  const int a = rp.acc_x ? rp.a : 0;
  const int nA = a + (rp.acc_y ? rp.b : 0);
  return nA >= 1 && nA <= OZ_MAXA;
}

int ozaki_gram_launch(const RowPass& rpin, Arena* ar, cudaStream_t st, int* launches, int num_sms) {
  RowPass rp = rpin;
  if (!rp.acc_x) { rp.a = 0; rp.X = nullptr; }
  if (!ozaki_gram_supported(rp) || rp.n <= 0) return RBO_ERR_ARG;
  const int a = rp.a, b = rp.b;
  const int nA = a + (rp.acc_y ? b : 0);
  const int N = ((8 * b + 15) / 16) * 16;
  const int zr = nA, no = zr * b, L = no;
  const int TP = OZ_T + 2;
  const size_t stage_bytes = (size_t)(a + b) * TP * 8;
  size_t o = 64;
  const size_t off_stage = o;
  o += NST * stage_bytes;
  const size_t off_tri = o;
  o += (size_t)b * b * 8;
  const size_t off_dinv = o;
  o += (size_t)b * 8;
  o = (o + 1023) & ~size_t(1023);
  const size_t off_B = o;
  o += (size_t)OZ_KS * N * 32;
  size_t epi = 64 + ((size_t)L + 2) * 8 + (size_t)b * b * 2 * 8 + 64 * 8;
  size_t comb = off_stage + (size_t)4 * OZ_MAXA * OZ_MAXB * 8;
  // at least 116 KB: one CTA per SM (each holds all 512 tensor-memory columns)
  size_t smem = std::max(std::max(o, epi), std::max(comb, (size_t)116 * 1024));
  if (smem > 220 * 1024) return RBO_ERR_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(g_oz_mu);
    if (dev >= 0 && dev < 64 && !g_oz_smem_set[dev]) {
      if (cudaFuncSetAttribute(ozaki_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               220 * 1024) != cudaSuccess)
        return note_cuda(cudaGetLastError());
      g_oz_smem_set[dev] = 1;
    }
  }
  const int ntiles = (int)((rp.n + OZ_T - 1) / OZ_T);
  int G = std::min(ntiles, std::max(num_sms, 1));
  if (rp.max_ctas > 0) G = std::min(G, rp.max_ctas);
  const int ngroups = (G + GROUP - 1) / GROUP;
  OzDev D;
  PassDev& P = D.P;
  P = PassDev();
  P.p = rp;
  P.T = OZ_T;
  P.TP = TP;
  P.ntiles = ntiles;
  const bool alignedX = a == 0 || (((uintptr_t)rp.X & 15) == 0 && (rp.ldx % 2) == 0);
  const bool alignedY = (((uintptr_t)rp.Y & 15) == 0 && (rp.ldy % 2) == 0);
  P.use_bulk = (alignedX && alignedY) ? 1 : 0;
  P.zr = zr;
  P.no = no;
  P.L = L;
  P.ngroups = ngroups;
  P.status = ar->status;
  P.off_stage = (int)off_stage;
  P.stage_bytes = (int)stage_bytes;
  P.off_tri = (int)off_tri;
  P.off_dinv = (int)off_dinv;
  P.off_red = 64;
  const size_t need = ((size_t)G * L + (size_t)ngroups * L) * 8;
  if (ar->red == nullptr || need > ar->red_bytes) return RBO_ERR_NOMEM;
  if (ngroups + 1 > ar->n_tickets) return RBO_ERR_NOMEM;
  P.partials = ar->red;
  P.gpart = ar->red + (size_t)G * L;
  P.tickets = ar->tickets;
  D.nA = nA;
  D.N = N;
  D.off_B = (int)off_B;
  ProfToken tok = prof_start(st);
  ozaki_gram_kernel<<<G, OZ_NT, smem, st>>>(D);
  if (prof_on()) {
    const double nn = (double)rp.n, A = a, B = b;
    const double by = 8.0 * nn * (A + B + (rp.write_y ? B : 0.0));
    double fl = 0.0;
    if (rp.Tri) fl += nn * B * B;
    if (rp.acc_x) fl += 2.0 * nn * A * B;
    if (rp.acc_y) fl += nn * B * (B + 1.0);
    prof_stop(tok, st, RBO_PROF_OZAKI, by, fl, rp.tag);
  }
  if (launches) ++*launches;
  return note_cuda(cudaGetLastError());
}

}  // namespace rbo

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
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "rowpass_common.cuh"

namespace rbo {
namespace {

constexpr int OZ_T = 128;            // rows per tile
constexpr int OZ_KS = OZ_T / 16;     // tensor-core K-steps per tile
constexpr int OZ_SPLIT = 256;        // splitter threads (two warpgroups)
constexpr int OZ_NT = OZ_SPLIT + 32; // and one warp issuing the tensor-core products
constexpr int OZ_RING = 8;           // K-step slots between splitters and the issuing warp
constexpr int OZ_TRING = 16;         // tile-completion barriers (> OZ_CHUNK)
constexpr int OZ_CHUNK = 8;          // tiles per accumulation chunk: 1024 rows, so every
                                     // digit-pair sum stays within 2^24 (exact in float32)
constexpr int OZ_HEAD = 1;           // a chunk's column scale: its first tile's exponent
                                     // maximum + OZ_HEAD ...
constexpr int OZ_WIN = 2;            // ... and later tiles join while their maxima stay
                                     // within [scale - OZ_WIN, scale]
constexpr int OZ_MAXA = 64;          // columns of [X Y'] in A
constexpr int OZ_MAXB = 8;           // columns of Y'
constexpr int OZ_GSTRIDE = 144;      // bytes per column of a K-step's fixed-point buffer
                                     // (16 rows of 8 bytes + 16: conflict-free 16-byte reads)
constexpr uint32_t OZ_TMEM_COLS = 512;
constexpr unsigned long long OZ_BIAS = 0x0080808080808080ULL;

struct OzDev {
  CUtensorMap tmX;   // X (n x a) and Y (n x b) as 2-D tensors: boxes of OZ_T rows x all
  CUtensorMap tmY;   // columns, rows past n read as zero
  PassDev P;
  int nA;      // columns of A: a (acc_x) then b (acc_y)
  int N;       // MMA N = 16 ceil(8 b / 16)
  int R;       // digits of a column side by side in the lanes: 2 (nA <= 64) or 4 (nA <= 32)
  int Q;       // A regions (one MMA each) per K-step: ceil(7 / R)
  int off_B;   // B slots: OZ_RING x N rows x 32 bytes
  int off_G;   // per warpgroup: fixed points of a K-step, (OZ_MAXA + OZ_MAXB) x OZ_GSTRIDE
};

// ---- PTX: tensor memory and the tensor-core MMA (tcgen05) ------------------------------
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // no-swizzle canonical layout: start >> 4, leading (K) byte offset >> 4, stride (M/N)
  // byte offset >> 4, descriptor version 1 (bits 46-48 = 0b001)
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}
// kind::f16 instruction descriptor: D float32, A and B fp16 (format 0), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (tensor memory) [+]= A (tensor memory) B (shared memory descriptor)
__device__ __forceinline__ void mma_f16(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
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
// one 2-D tile of a tensor map into shared memory (rows x0.., columns 0..), completion
// counted on `bar`
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x0, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x0), "r"(0), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- digits -----------------------------------------------------------------------------
// F = y 2^(1076 - E) rounded to nearest (ties away from zero); |F| < 2^54 for a value
// whose exponent field is at most E (E >= 1); zero and subnormal values give 0.
__device__ __forceinline__ long long oz_fix(double y, int E) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(y);
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long M = (u & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const int k = E - 1 - e;  // right shift; -1 when e == E
  unsigned long long v;
  if (k < 0) v = M << 1;
  else if (k < 63) v = (M + ((1ULL << k) >> 1)) >> k;
  else v = 0;
  if (e == 0) v = 0;
  return (u >> 63) ? -(long long)v : (long long)v;
}
// the biased fixed point G = F + 0x0080808080808080 as two words
struct G2 {
  uint32_t lo, hi;
};
// G of y for the column scale exponent E (every value of the column in the chunk has
// an exponent field <= E): F = round(y 2^(1073 - E)), |F| < 2^51.  Integer operations
// only: y = +-M 2^(e - 1075) (M the 53-bit significand), so F = +-round(M 2^-(E + 2 - e)),
// a right shift by k = E + 2 - e >= 2 with the rounding bit added first (ties away
// from zero).  Zero and subnormal values give F = 0.
__device__ __forceinline__ unsigned long long int_g(unsigned long long ub, int E) {
  const int e = (int)((ub >> 52) & 0x7FF);
  const unsigned long long M = (ub & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const int k = E + 2 - e;
  unsigned long long r = k < 64 ? (M + (1ULL << (k - 1))) >> k : 0ULL;
  if (e == 0) r = 0ULL;
  return (ub >> 63) ? OZ_BIAS - r : OZ_BIAS + r;
}
__device__ __forceinline__ G2 biased_fix(double v, int E) {
  const unsigned long long g = (unsigned long long)oz_fix(v, E) + OZ_BIAS;
  return G2{(uint32_t)g, (uint32_t)(g >> 32)};
}
// Digit I = 6 - K of two values (byte K of their G, minus 128) as an fp16 pair: the two
// bytes placed in the low bytes of the halves of 1024 (0x6400), minus 1152 = 1024 + 128
// (both exact in fp16); x in the low half.
template <int K>
__device__ __forceinline__ uint32_t digit_pair(G2 x, G2 y) {
  constexpr uint32_t kk = K & 3;
  constexpr uint32_t sel = kk | (kk << 4) | ((4 + kk) << 8) | ((4 + kk) << 12);
  const uint32_t t = __byte_perm(K >= 4 ? x.hi : x.lo, K >= 4 ? y.hi : y.lo, sel);
  const uint32_t u = (t & 0x00FF00FFu) | 0x64006400u;
  const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&u),
                            __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));
  return *reinterpret_cast<const uint32_t*>(&h);
}

// A digits of one column for the 16 rows of a K-step from its fixed points gc (16 x 8
// bytes): digits I = q R + RHO of region q, row pairs packed, w[8 q + j]
template <int R, int RHO>
__device__ __forceinline__ void digits_a(const unsigned char* gc, uint32_t* w) {
  constexpr int Q = (7 + R - 1) / R;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint4 pr = *reinterpret_cast<const uint4*>(gc + 16 * j);
    const G2 g0{pr.x, pr.y}, g1{pr.z, pr.w};
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int I = q * R + RHO;
      if (I == 0) w[q * 8 + j] = digit_pair<6>(g0, g1);
      else if (I == 1) w[q * 8 + j] = digit_pair<5>(g0, g1);
      else if (I == 2) w[q * 8 + j] = digit_pair<4>(g0, g1);
      else if (I == 3) w[q * 8 + j] = digit_pair<3>(g0, g1);
      else if (I == 4) w[q * 8 + j] = digit_pair<2>(g0, g1);
      else if (I == 5) w[q * 8 + j] = digit_pair<1>(g0, g1);
      else if (I == 6) w[q * 8 + j] = digit_pair<0>(g0, g1);
      else w[q * 8 + j] = 0u;
    }
  }
}
// the same for a byte index k known only at run time (the selector is a register)
__device__ __forceinline__ uint32_t digit_pair_rt(G2 x, G2 y, int k) {
  const uint32_t kk = (uint32_t)(k & 3);
  const uint32_t sel = kk * 0x1111u + 0x4400u;  // bytes kk, kk of x; kk, kk of y
  const bool h = k >= 4;
  const uint32_t t = __byte_perm(h ? x.hi : x.lo, h ? y.hi : y.lo, sel);
  const uint32_t u = (t & 0x00FF00FFu) | 0x64006400u;
  const __half2 r = __hsub2(*reinterpret_cast<const __half2*>(&u),
                            __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));
  return *reinterpret_cast<const uint32_t*>(&r);
}
// bounded wait (mbarrier.try_wait suspends the thread for a while between polls);
// false on timeout
__device__ __forceinline__ bool wait_backoff(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

// ---- the kernel ---------------------------------------------------------------------------
// Roles: warps 0-7 (two warpgroups) split tiles into digits; warpgroup wg produces the
// K-steps ks = wg, wg + 2, ... of each tile into a ring of OZ_RING slots (A: tensor
// memory, B: shared memory) and hands each to warp 8, whose lane 0 issues the
// tensor-core products (mbarriers full / empty per slot).  The accumulators D stay in
// tensor memory over a chunk of up to OZ_CHUNK tiles that share one scale per column
// (the first tile's exponent maximum plus OZ_HEAD): a tile whose exponents exceed the
// chunk's scale, or a full chunk, starts a new chunk after the splitters drained D into
// 128-bit integer accumulators.
__global__ void __launch_bounds__(OZ_NT, 1) ozaki_gram_kernel(const __grid_constant__ OzDev D) {
  const PassDev& P = D.P;
  const RowPass& rp = P.p;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // offsets are taken from a 1024-byte aligned base (the launch adds 1 KB of slack):
  // tensor copies and the tensor-core operand descriptors need aligned addresses
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ int s_flag;
  __shared__ int s_last;
  __shared__ uint32_t s_tmem;
  __shared__ int s_Et[OZ_MAXA + OZ_MAXB];   // exponent field maximum per column, this tile
  __shared__ int s_Ec[OZ_MAXA + OZ_MAXB];   // column scale exponents of the open chunk
  __shared__ int s_bad[OZ_MAXA + OZ_MAXB];  // a non-finite value met in the column
  __shared__ int s_exceed, s_abort;
  __shared__ int s_wgfail[2];
  __shared__ int s_slot_start[OZ_RING];     // K-step in the slot starts a chunk
  __shared__ __align__(8) uint64_t s_full[OZ_RING];
  __shared__ __align__(8) uint64_t s_empty[OZ_RING];
  __shared__ __align__(8) uint64_t s_tile[OZ_TRING];
  __shared__ __align__(8) uint64_t s_final;
  if (read_code(P.status) != 0) return;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool splitter = tid < OZ_SPLIT;
  const int wg = warp >> 2;  // 0, 1 (2 for the issuing warp)
  const int a = rp.a, b = rp.b, T = OZ_T, TP = P.TP;
  const int ncol = a + b;
  const int nA = D.nA, N = D.N, R = D.R, Q = D.Q;
  const int64_t n = rp.n;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  double* Ts = reinterpret_cast<double*>(smem + P.off_tri);
  double* dinv = reinterpret_cast<double*>(smem + P.off_dinv);
  unsigned char* Bs = smem + D.off_B;
  auto bar_split = []() { asm volatile("bar.sync 1, 256;" ::: "memory"); };
  const int wg_bar = 2 + wg;
  auto bar_wg = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(wg_bar) : "memory"); };

  if (rp.Tri) {
    const int ldt = rp.ldtri > 0 ? rp.ldtri : b;
    for (int t = tid; t < b * b; t += OZ_NT) {
      const int i = t % b, c = t / b;
      Ts[t] = (i <= c) ? rp.Tri[i + (size_t)c * ldt] : 0.0;
    }
    for (int t = tid; t < b; t += OZ_NT) dinv[t] = 1.0 / rp.Tri[t + (size_t)t * ldt];
  }
  // B slots: rows 8 yc + 7 and rows >= 8 b stay zero
  for (int t = tid; t < OZ_RING * N * 8; t += OZ_NT) reinterpret_cast<uint32_t*>(Bs)[t] = 0u;
  for (int t = tid; t < OZ_MAXA + OZ_MAXB; t += OZ_NT) {
    s_bad[t] = 0;
    s_Ec[t] = 0;
  }
  if (tid == 0) {
    s_abort = 0;
    s_wgfail[0] = s_wgfail[1] = 0;
    for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
    for (int s = 0; s < OZ_RING; ++s) {
      mbar_init(&s_full[s], 4);
      mbar_init(&s_empty[s], 1);
    }
    for (int s = 0; s < OZ_TRING; ++s) mbar_init(&s_tile[s], 1);
    mbar_init(&s_final, 1);
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
  const uint32_t tA = s_tmem;                    // A ring: slot s at columns 32 s, region q at + 8 q
  const uint32_t tD = s_tmem + 32 * OZ_RING;     // D_q at columns 32 OZ_RING + q N
  const int first = blockIdx.x;
  const int ntl = first < P.ntiles ? (P.ntiles - first + (int)gridDim.x - 1) / (int)gridDim.x : 0;

  // ======================= tensor-core issue (warp 8, lane 0) =============================
  if (!splitter) {
    if (lane == 0) {
      const uint32_t id = idesc_f16(128, N);
      bool ok = true;
      for (int it = 0; it < ntl && ok; ++it) {
        for (int ks = 0; ks < OZ_KS; ++ks) {
          const int g = it * OZ_KS + ks, slot = g % OZ_RING;
          if (!wait_backoff(&s_full[slot], (uint32_t)((g / OZ_RING) & 1))) {
            set_error(P.status, RBO_ERR_TIMEOUT, 13);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = s_slot_start[slot] ? 0u : 1u;
          const uint64_t db = smem_desc(smem_u32(Bs + (size_t)slot * N * 32), 128, 256);
          for (int q = 0; q < Q; ++q)
            mma_f16(tD + (uint32_t)(q * N), tA + (uint32_t)(32 * slot + 8 * q), db, id, acc);
          mma_commit(&s_empty[slot]);
        }
        if (ok) mma_commit(&s_tile[it % OZ_TRING]);
      }
      // every product issued has completed before the tensor memory is freed
      mma_commit(&s_final);
      mbar_wait_bounded(&s_final, 0u);
    }
  } else {
    // ======================= splitters (warps 0-7) =========================================
    const int wq = warp & 3;
    const int L = 32 * wq + lane;                 // this thread's A lane
    const int rho = R == 2 ? (wq >> 1) : wq;      // digit group (warp-uniform)
    const int xc = R == 2 ? (L & 63) : lane;      // A column
    const bool active = xc < nA;
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
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
    // a tile: two tensor copies (X box, Y box) issued by one thread
    auto issue_tile = [&](int tile, int s) {
      if (lane != 0) return;
      const int r0 = tile * T;
      double* xs = stage_X(s);
      mbar_arrive_expect_tx(&bars[s], (uint32_t)T * 8u * (uint32_t)ncol);
      if (a > 0) tma_load_2d(xs, &D.tmX, r0, &bars[s]);
      tma_load_2d(xs + (size_t)a * TP, &D.tmY, r0, &bars[s]);
    };
    // drain D (all products of the open chunk complete) into the 128-bit accumulators
    auto drain = [&]() {
      long long hi[OZ_MAXB], lo[OZ_MAXB];
#pragma unroll
      for (int c = 0; c < OZ_MAXB; ++c) { hi[c] = 0; lo[c] = 0; }
      const int q0 = wg * (Q / 2), q1 = q0 + Q / 2;
      for (int q = q0; q < q1; ++q) {
        const int I = q * R + rho;
#pragma unroll
        for (int yc = 0; yc < OZ_MAXB; ++yc) {
          if (yc < b) {  // b is uniform: the loads stay warp-converged
            float v[8];
            tmem_ld8(tD + (uint32_t)(q * N + 8 * yc) + lane_base, v);
            if (active && I <= 6) {
#pragma unroll
              for (int J = 0; J < 7; ++J) {
                const int Lv = I + J;
                if (Lv <= 7) {
                  const long long iv = (long long)__float2int_rn(v[J]);
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
              const int Tt = s_Ec[xc] + s_Ec[a + yc];
              if (ea[yc] < 0) ea[yc] = Tt;
              int sh = Tt - ea[yc];
              // |S| < 2^83; a shift of at most 20 keeps the sum of the CTA's chunks far
              // below 2^127
              if (sh > 20) {
                acc[yc] >>= (sh - 20);
                ea[yc] += sh - 20;
                sh = 20;
              }
              if (sh >= 0) acc[yc] += S << sh;
              else if (sh > -120) acc[yc] += S >> (-sh);
            }
          }
        }
      }
    };

    uint32_t phase[NST] = {0u, 0u};
    bool chunk_open = false;
    int tiles_in_chunk = 0;
    if (ntl > 0 && warp == 0) issue_tile(first, 0);
    int it = 0;
    for (; it < ntl; ++it) {
      const int tile = first + it * (int)gridDim.x;
      const int s = it & 1;
      const int64_t r0 = (int64_t)tile * T;
      const int rows = (n - r0 < (int64_t)T) ? (int)(n - r0) : T;
      double* xs = stage_X(s);
      double* ys = xs + (size_t)a * TP;
      if (tid == 0) s_exceed = 0;
      {
        const bool ok = wait_backoff(&bars[s], phase[s]);
        if (!__all_sync(0xffffffffu, ok) && lane == 0) {
          set_error(P.status, RBO_ERR_TIMEOUT, 11);
          s_abort = 1;
        }
        phase[s] ^= 1u;
      }
      bar_split();
      if (s_abort) break;
      if (it + 1 < ntl && warp == 0) {
        fence_proxy_async();
        issue_tile(tile + (int)gridDim.x, s ^ 1);
      }

      // ---- y' = y Tri^-1 (float64), written back ----------------------------------------
      if (rp.Tri) {
        for (int c0 = 0; c0 < b; c0 += CB) {
          const int cw = min(CB, b - c0);
          if (c0 > 0) {
            for (int t = tid; t < T * cw; t += OZ_SPLIT) {
              const int r = t % T, c = c0 + t / T;
              double v = ys[c * TP + r];
              for (int i = 0; i < c0; ++i) v = fma(-ys[i * TP + r], Ts[i + c * b], v);
              ys[c * TP + r] = v;
            }
            bar_split();
          }
          for (int r = tid; r < T; r += OZ_SPLIT) {
            for (int c = c0; c < c0 + cw; ++c) {
              double v = ys[c * TP + r];
              for (int i = c0; i < c; ++i) v = fma(-ys[i * TP + r], Ts[i + c * b], v);
              ys[c * TP + r] = v * dinv[c];
            }
          }
          bar_split();
        }
        if (rp.write_y)
          for (int t = tid; t < b * T; t += OZ_SPLIT) {
            const int c = t / T, rr = t % T;
            if (rr < rows) rp.Y[c * rp.ldy + r0 + rr] = ys[(size_t)c * TP + rr];
          }
        fence_proxy_async();  // the stage was written here; a later tensor copy reuses it
      }

      // ---- exponent field maxima; a new chunk when they exceed the chunk's scales -------
      // one warp per column (columns warp, warp + 8, ...): every load first, four rows
      // per lane and column, then the warp maxima
      {
        constexpr int NCW = (OZ_MAXA + OZ_MAXB) / (OZ_SPLIT / 32);
        uint32_t m[NCW];
#pragma unroll
        for (int i = 0; i < NCW; ++i) {
          const int c = warp + 8 * i;
          m[i] = 0u;
          if (c < ncol) {
            const uint32_t* col = reinterpret_cast<const uint32_t*>(xs + (size_t)c * TP);
#pragma unroll
            for (int k = 0; k < T / 32; ++k) m[i] = max(m[i], col[2 * (32 * k + lane) + 1] & 0x7FFFFFFFu);
          }
        }
#pragma unroll
        for (int i = 0; i < NCW; ++i) {
          const int c = warp + 8 * i;
          const uint32_t e = __reduce_max_sync(0xffffffffu, (m[i] >> 20) & 0x7FFu);
          if (lane == 0 && c < ncol) s_Et[c] = (int)e;
        }
      }
      bar_split();
      for (int c = tid; c < ncol; c += OZ_SPLIT) {
        // outside the chunk's window: larger values would overflow its fixed point,
        // much smaller ones would lose bits (a column of zeros fits every window)
        if (s_Et[c] > s_Ec[c] || (s_Et[c] != 0 && s_Et[c] < s_Ec[c] - OZ_WIN)) s_exceed = 1;
        if (s_Et[c] == 0x7FF) s_bad[c] = 1;
      }
      bar_split();
      const bool new_chunk = !chunk_open || tiles_in_chunk == OZ_CHUNK || s_exceed;
      if (new_chunk) {
        if (chunk_open) {
          const int pt = it - 1;
          const bool ok = wait_backoff(&s_tile[pt % OZ_TRING], (uint32_t)((pt / OZ_TRING) & 1));
          if (!__all_sync(0xffffffffu, ok) && lane == 0) {
            set_error(P.status, RBO_ERR_TIMEOUT, 14);
            s_abort = 1;
          }
          bar_split();
          if (s_abort) break;
          tc_fence_after();
          drain();
          tc_fence_before();
        }
        bar_split();
        for (int c = tid; c < ncol; c += OZ_SPLIT) s_Ec[c] = s_Et[c] + OZ_HEAD;
        bar_split();
        chunk_open = true;
        tiles_in_chunk = 0;
      }
      ++tiles_in_chunk;

      // ---- digits of this warpgroup's K-steps: A into tensor memory, B into shared ------
      // Per K-step: (1) the 128 threads of the warpgroup form the biased fixed point of
      // every value of the 16 rows (each value once) in the warpgroup's buffer; (2) each
      // A lane reads its column's 16 values and packs its digits; the B tasks pack the
      // Y' digits.
      bool fail = false;
      const int t128 = tid & 127;
      unsigned char* gb = smem + D.off_G + (size_t)wg * (OZ_MAXA + OZ_MAXB) * OZ_GSTRIDE;
      for (int ks = wg; ks < OZ_KS; ks += 2) {
        const int g = it * OZ_KS + ks, slot = g % OZ_RING;
        {
          const int r = t128 & 15;
          const int c0 = t128 >> 4;
          constexpr int NCI = (OZ_MAXA + OZ_MAXB) / 8;
          unsigned long long u[NCI];
          int E[NCI];
#pragma unroll
          for (int i = 0; i < NCI; ++i) {  // every load first
            const int c = c0 + 8 * i;
            u[i] = c < ncol ? (unsigned long long)__double_as_longlong(xs[(size_t)c * TP + ks * 16 + r]) : 0ULL;
            E[i] = c < ncol ? s_Ec[c] : 0;
          }
#pragma unroll
          for (int i = 0; i < NCI; ++i) {
            const int c = c0 + 8 * i;
            if (c < ncol)
              *reinterpret_cast<unsigned long long*>(gb + (size_t)c * OZ_GSTRIDE + r * 8) = int_g(u[i], E[i]);
          }
        }
        // the slot's previous products have completed (its A and B may be overwritten)
        const bool ok = g < OZ_RING || wait_backoff(&s_empty[slot], (uint32_t)(((g / OZ_RING) - 1) & 1));
        if (!ok) {
          set_error(P.status, RBO_ERR_TIMEOUT, 15);
          s_wgfail[wg] = 1;
        }
        bar_wg();
        if (s_wgfail[wg]) {  // uniform in the warpgroup
          fail = true;
          break;
        }
        tc_fence_after();
        uint32_t w[32];
#pragma unroll
        for (int j2 = 0; j2 < 32; ++j2) w[j2] = 0u;
        if (active) {
          const unsigned char* gc = gb + (size_t)xc * OZ_GSTRIDE;
          if (R == 2) {
            if (rho == 0) digits_a<2, 0>(gc, w);
            else digits_a<2, 1>(gc, w);
          } else {
            switch (rho) {
              case 0: digits_a<4, 0>(gc, w); break;
              case 1: digits_a<4, 1>(gc, w); break;
              case 2: digits_a<4, 2>(gc, w); break;
              default: digits_a<4, 3>(gc, w); break;
            }
          }
        }
        if (R == 2) tmem_st32(tA + (uint32_t)(32 * slot) + lane_base, w);
        else tmem_st16(tA + (uint32_t)(32 * slot) + lane_base, w);
        // B: Y' digits, row 8 yc + J of the K-major slot, one digit pair per task
        unsigned char* Bk = Bs + (size_t)slot * N * 32;
        if (t128 < 8 * b) {
          const int jp = t128 & 7, yc = t128 >> 3;
          const uint4 pr = *reinterpret_cast<const uint4*>(gb + (size_t)(a + yc) * OZ_GSTRIDE + 16 * jp);
          const G2 g0{pr.x, pr.y}, g1{pr.z, pr.w};
          uint32_t* dst = reinterpret_cast<uint32_t*>(Bk + yc * 256 + (jp >> 2) * 128 + (jp & 3) * 4);
          dst[0] = digit_pair<6>(g0, g1);   // rows 8 yc + J are 16 bytes apart
          dst[4] = digit_pair<5>(g0, g1);
          dst[8] = digit_pair<4>(g0, g1);
          dst[12] = digit_pair<3>(g0, g1);
          dst[16] = digit_pair<2>(g0, g1);
          dst[20] = digit_pair<1>(g0, g1);
          dst[24] = digit_pair<0>(g0, g1);
        }
        if (t128 == 0) s_slot_start[slot] = (new_chunk && ks == 0) ? 1 : 0;
        tmem_wait_st();
        if (t128 < 8 * b) fence_proxy_async();  // B written through the generic proxy
        tc_fence_before();
        bar_wg();  // the buffer is free for the next K-step; the slot is complete
        if (lane == 0) mbar_arrive(&s_full[slot]);
      }
      if (fail) s_abort = 1;
      bar_split();  // stage s free; every K-step of the tile handed over
      if (s_abort) break;
    }
    // ---- the last chunk ------------------------------------------------------------------
    if (!s_abort && chunk_open && it == ntl) {
      const int pt = ntl - 1;
      const bool ok = wait_backoff(&s_tile[pt % OZ_TRING], (uint32_t)((pt / OZ_TRING) & 1));
      if (!__all_sync(0xffffffffu, ok) && lane == 0) {
        set_error(P.status, RBO_ERR_TIMEOUT, 14);
        s_abort = 1;
      }
      bar_split();
      if (!s_abort) {
        tc_fence_after();
        drain();
      }
    }
    bar_split();
    // per-CTA partial contributions: (warpgroup, digit group) slot of every output
    double* comb = reinterpret_cast<double*>(smem + P.off_stage);  // 8 x 64 x 8
    const int cslot = wg * 4 + rho;
    if (!s_abort)
      for (int t = tid; t < 8 * OZ_MAXA * OZ_MAXB; t += OZ_SPLIT) comb[t] = 0.0;
    bar_split();
    if (!s_abort && active) {
#pragma unroll
      for (int yc = 0; yc < OZ_MAXB; ++yc) {
        if (yc < b && ea[yc] >= 0)
          comb[((size_t)cslot * OZ_MAXA + xc) * OZ_MAXB + yc] = ldexp((double)acc[yc], ea[yc] - 2106);
      }
    }
  }

  // ---- free the tensor memory (every issued product has completed) -------------------------
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && read_code(P.status) != 0) s_abort = 1;
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem),
                 "r"(OZ_TMEM_COLS));
  }
  __syncthreads();
  if (s_abort || P.L == 0) return;

  const double* comb = reinterpret_cast<const double*>(smem + P.off_stage);
  double* mypart = P.partials + (size_t)blockIdx.x * P.L;
  for (int o = tid; o < P.no; o += OZ_NT) {
    const int i = o / b, c = o % b;
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += comb[((size_t)k * OZ_MAXA + i) * OZ_MAXB + c];
    if (s_bad[i] || s_bad[a + c]) sum = __longlong_as_double(0x7FF8000000000000LL);
    mypart[o] = sum;
  }
  tree_reduce_epilogue(P, smem, &s_flag, &s_last);
}

std::mutex g_oz_mu;
int g_oz_smem_set[64] = {};

}  // namespace

// 2-D tensor map of a column-major float64 array (n rows, cols columns, leading
// dimension ld): boxes of OZ_T rows x cols columns, out-of-range rows read as zero.
static int make_tensor_map(CUtensorMap* m, const double* base, int64_t n, int cols, int64_t ld) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_oz_mu);
    if (encode == nullptr) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
              cudaSuccess ||
          q != cudaDriverEntryPointSuccess || fn == nullptr) {
        cudaGetLastError();
        return RBO_ERR_CUDA;
      }
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)cols};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  const cuuint32_t box[2] = {(cuuint32_t)OZ_T, (cuuint32_t)cols};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims,
                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RBO_OK : RBO_ERR_CUDA;
}

bool ozaki_gram_supported(const RowPass& rp) {
  if (!rp.ozaki || rp.C || rp.sk_d > 0 || rp.sk_gd > 0 || rp.mixed || rp.df64) return false;
  if (!rp.acc_x && !rp.acc_y) return false;
  if (rp.b < 1 || rp.b > OZ_MAXB) return false;
  const int a = rp.acc_x ? rp.a : 0;
  // tensor copies: 16-byte aligned bases and column strides, row coordinates in int
  if (rp.n >= (int64_t)1 << 31) return false;
  if (((uintptr_t)rp.Y & 15) != 0 || (rp.ldy % 2) != 0) return false;
  if (a > 0 && (((uintptr_t)rp.X & 15) != 0 || (rp.ldx % 2) != 0)) return false;
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
  const int TP = OZ_T;  // the tensor copies fill columns of exactly OZ_T rows
  const size_t stage_bytes = (size_t)(a + b) * TP * 8;
  size_t o = 1024;       // tensor-copy destinations 128-byte aligned
  const size_t off_stage = o;
  o += NST * stage_bytes;
  const size_t off_tri = o;
  o += (size_t)b * b * 8;
  const size_t off_dinv = o;
  o += (size_t)b * 8;
  o = (o + 1023) & ~size_t(1023);
  const size_t off_B = o;
  o += (size_t)OZ_RING * N * 32;
  const size_t off_G = o;
  o += (size_t)2 * (OZ_MAXA + OZ_MAXB) * OZ_GSTRIDE;
  size_t epi = 64 + ((size_t)L + 2) * 8 + (size_t)b * b * 2 * 8 + 64 * 8;
  size_t comb = off_stage + (size_t)8 * OZ_MAXA * OZ_MAXB * 8;
  // at least 116 KB: one CTA per SM (each holds all 512 tensor-memory columns)
  size_t smem = std::max(std::max(o, epi), std::max(comb, (size_t)116 * 1024));
  smem += 1024;  // alignment slack of the kernel's base
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
  P.use_bulk = 1;
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
  D.R = nA <= 32 ? 4 : 2;
  D.Q = (7 + D.R - 1) / D.R;
  D.off_B = (int)off_B;
  D.off_G = (int)off_G;
  {
    int e = make_tensor_map(&D.tmY, rp.Y, rp.n, b, rp.ldy);
    if (e == RBO_OK && a > 0) e = make_tensor_map(&D.tmX, rp.X, rp.n, a, rp.ldx);
    if (e != RBO_OK) return e;
  }
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

// Tensor-core Gram pass: Z = [X Y]^T Y with float64 accuracy from exact products of
// 8-bit digits on the fp16 tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// The Gram matrices of BCGS and CholQR (Sections 4-5, the reductions Q^T W and W^T W)
// are the float64 contractions of the method.  On this GPU the float64 pipe (2 FMA per
// SM per clock) caps a float64 Gram pass near 1.1 TFLOP/s, far below the HBM rate, while
// the fp16 tensor cores are three orders of magnitude faster.  Splitting every float64
// value into digits that fp16 represents exactly turns the Gram into exact integer
// products (the idea of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59, 2012):
//
//   * the rows are cut into tiles of 128 and the tiles of a CTA into accumulation chunks
//     of at most 8 tiles (1024 rows); per chunk and column c a scale exponent E_c, at
//     least every exponent field of the column in the chunk: the first tile's largest
//     exponent field plus one, later tiles joining while their largest field stays in
//     [E_c - 2, E_c];
//   * every value becomes the integer F = sign * (M >> (E_c - e)) (M its 53-bit
//     significand, e its exponent field), |F| < 2^53, an error below 2^-50 of the
//     column's largest magnitude in the tile; zero and subnormal values give 0;
//   * G = F + 0x0080808080808080 lies in [0, 2^56); byte k of G minus 128 is the
//     balanced digit d_k in [-128, 127] with F = sum_k d_k 2^(8k); digit I = 0..6 is
//     byte 6 - I (most significant first), each exact in fp16;
//   * a product of two digits is an integer of at most 2^14 in magnitude, so a sum over
//     the 1024 rows of a chunk stays within 2^24: exact in the float32 accumulator
//     whatever the order of the additions;
//   * the digit pairs (I, J) with I + J <= 7 are kept (the dropped ones weigh less than
//     2^-57 of the product of the two columns' largest magnitudes); per chunk they are
//     combined in 64-bit integers and added, shifted by the chunk's exponents, into a
//     128-bit integer accumulator per output; the per-CTA value is rounded to float64
//     once per (warpgroup, digit parity) and the four roundings summed.
//
// Tensor-core mapping (M = 128, K = 16 rows per instruction):
//   A (tensor memory): lane (c, p) = column c of [X Y] (c < 64) with digits of parity p;
//     region q = 0..3 of a K-step holds digit I = 2q + p (I = 7: no digit, ignored);
//   B (shared memory, no-swizzle K-major): row 8 yc + J = digit J of column yc of Y;
//   D_q (tensor memory, one region per q): D_q[(c, p), 8 yc + J] = sum over the chunk's
//     rows of digit (2q + p) of x_c times digit J of y_yc.
// Per K-step four instructions; the regions are independent accumulators.
//
// Work split: one warp issues the tensor copies of the row tiles; one warp scans each
// landed tile for its columns' exponent maxima and takes the chunk decisions (a record
// per stage: new chunk or not, the scale of every column); two warpgroups of splitters
// (warpgroup wg takes the K-steps wg, wg + 2, ... of every tile) write the digits; one
// warp issues the tensor-core products.  A splitter thread owns one column and one half
// (8 rows) of each of its K-steps: it forms the fixed points of its 8 values, packs their
// digit bytes for itself and for the lane holding the other half of the column, swaps
// the packed words with that lane, and writes the 16 rows' digits of its parity into
// the tensor memory; the threads of Y columns also store those digit words as the B
// operand.  No named barrier is used inside the tile loop: every handshake is an
// mbarrier with a bounded wait, and a thread that gives up makes every other wait of the
// CTA give up too.
//
// Supported passes: Gram of [X Y]^T Y (acc_x and/or acc_y) with a + b <= 64 columns,
// b <= 8.  Everything after the per-CTA partials (the fixed-order tree and the small
// dense epilogue) is shared with the float64 row pass.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "rowpass_common.cuh"

namespace rbo {
namespace {

constexpr int OZ_T = 128;              // rows per tile
constexpr int OZ_KS = OZ_T / 16;       // tensor-core K-steps per tile (= ring slots)
constexpr int OZ_KPW = OZ_KS / 2;      // K-steps per splitter thread and tile
constexpr int OZ_SPLIT = 256;          // splitter threads (two warpgroups)
constexpr int OZ_NT = OZ_SPLIT + 96;   // + the issuing, copy and scanning warps
constexpr int OZ_MMA_WARP = 8;
constexpr int OZ_TMA_WARP = 9;
constexpr int OZ_SCAN_WARP = 10;
constexpr int OZ_TRING = 16;           // tile-completion barriers (> OZ_CHUNK)
constexpr int OZ_CHUNK = 8;            // tiles per accumulation chunk: 1024 rows
constexpr int OZ_HEAD = 1;             // chunk scale = first tile's exponent maximum + 1
constexpr int OZ_WIN = 2;              // later tiles join while within [scale - 2, scale]
constexpr int OZ_MAXA = 64;            // columns of [X Y] in A
constexpr int OZ_MAXB = 8;             // columns of Y
constexpr int OZ_MAXST = 8;            // row-tile stages
constexpr uint32_t OZ_TMEM_COLS = 512;
constexpr unsigned long long OZ_BIAS = 0x6480808080808080ULL;  // digit bias + fp16 exponent byte

struct OzDev {
  CUtensorMap tmX;   // X (n x a) and Y (n x b): boxes of 16 rows x all columns, 128-byte
  CUtensorMap tmY;   // swizzle, rows past n read as zero
  PassDev P;
  int nA;            // columns of A: a + b
  int zr;            // Z rows written: a (acc_x) then b (acc_y)
  int N;             // MMA N = 16 ceil(8 b / 16)
  int nst;           // row-tile stages
  int xbox, ybox;    // bytes of one K-step box of X, of Y (multiples of 1024)
  int stage_bytes;   // 8 (xbox + ybox)
  int off_B;         // B slots: OZ_KS x N rows x 32 bytes
};

// ---- PTX: tensor memory, tensor copies and the tensor-core MMA (tcgen05) ----------------
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
// one 2-D box of a tensor map into shared memory (rows x0.., columns 0..), completion
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
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 8 columns of this warp's lane quarter; the wait is in the same statement
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
// named barrier 1 over the 256 splitter threads
__device__ __forceinline__ void bar_split() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// ---- digits -----------------------------------------------------------------------------
// The biased fixed point G = F + 0x6480808080808080 (as two words) of the float64 value
// with bits (lo, hi) at the column scale exponent Ec (every exponent field of the column
// in the chunk is at most Ec): F = sign * (M >> (Ec - e)) with M the 53-bit significand
// and e the exponent field, |F| < 2^53.  Bytes 0-6 of F + 0x0080808080808080 are the
// biased balanced digits; byte 7 is 0x64, the high byte of the fp16 1024 that turns a
// digit byte into an fp16 value (see oz_digits).  Integer operations only: a shift by
// 32 when Ec - e >= 32, a funnel shift, and the sign applied as (r ^ s) - s with s = 0
// or -1.  CAREFUL: zero and subnormal values (e = 0) give F = 0 for any Ec; without it
// that holds only for Ec >= 64 (a shift of 63 leaves nothing of M), the case of every
// column whose largest magnitude is above 2^-959.
template <bool CAREFUL>
__device__ __forceinline__ void oz_fix(uint32_t lo, uint32_t hi, int Ec, uint32_t& gl, uint32_t& gh) {
  const int e = (int)((hi >> 20) & 0x7FFu);
  int k = min(Ec - e, 63);
  if (CAREFUL && e == 0) k = 63;
  const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
  const bool big = k >= 32;
  const uint32_t l = big ? mh : lo;
  const uint32_t h = big ? 0u : mh;
  const uint32_t rl = __funnelshift_r(l, h, (uint32_t)k);  // shift count taken mod 32
  const uint32_t rh = h >> (k & 31);
  const uint32_t s = (uint32_t)((int)hi >> 31);
  const unsigned long long x = ((unsigned long long)(rh ^ s) << 32) | (unsigned long long)(rl ^ s);
  const unsigned long long g = x + OZ_BIAS + (unsigned long long)(hi >> 31);
  gl = (uint32_t)g;
  gh = (uint32_t)(g >> 32);
}
// The fp16 pair of the digits held in bytes (0, 2) or (2, 3) of two packed words: a
// packed word of a row holds [digit byte, 0x64, digit byte, 0x64], i.e. two fp16 values
// 1024 + byte; the pair takes one of them from each row (x: row 2j, y: row 2j + 1) and
// subtracts 1152 = 1024 + 128 (all exact in fp16).
__device__ __forceinline__ uint32_t oz_digits(uint32_t x, uint32_t y, uint32_t sel) {
  const uint32_t t = __byte_perm(x, y, sel);
  const __half2 h = __hsub2(*reinterpret_cast<const __half2*>(&t),
                            __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));
  return *reinterpret_cast<const uint32_t*>(&h);
}
// non-blocking test of an mbarrier phase
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait that gives up at once when another thread of the CTA has given up
// (`abort` set); a timeout sets `abort`
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// ---- the kernel ---------------------------------------------------------------------------
// Handshakes (all mbarriers, every wait bounded):
//   stage full / ready / empty: the tensor copies of a tile have landed / the scanner
//     has published the tile's record / the 8 splitter warps are done with the stage;
//   K-step slot full / empty (slot = K-step index in the tile): the 4 warps of the owning
//     warpgroup have written A (tensor memory) and B (shared memory) / the products of
//     the slot have completed (tcgen05.commit);
//   tile: every product of the tile has completed (before a chunk's accumulators are
//     drained); drained: the 8 splitter warps have read the accumulators (before the
//     next chunk's first products overwrite them).
// A chunk's accumulators are drained by the splitters (regions 0-1 by warpgroup 0, 2-3
// by warpgroup 1) into 128-bit integer accumulators per (thread, Y column).
__global__ void __launch_bounds__(OZ_NT, 1) ozaki_gram_kernel(const __grid_constant__ OzDev D) {
  const PassDev& P = D.P;
  const RowPass& rp = P.p;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // offsets are taken from a 1024-byte aligned base (the launch adds 1 KB of slack): the
  // 128-byte swizzle of the tensor copies repeats every 1024 bytes
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ int s_flag, s_last, s_skip, s_aborted;
  __shared__ volatile int s_abort;    // some wait gave up
  __shared__ volatile int s_issued;   // tiles whose copies were issued
  __shared__ volatile int s_landed;   // tiles the scanner saw land
  __shared__ uint32_t s_tmem;
  __shared__ int s_bad[OZ_MAXA];                // a non-finite value met in the column
  __shared__ int s_rec_newc[OZ_MAXST];          // stage record: the tile starts a chunk,
  __shared__ int s_rec_careful[OZ_MAXST];       // a column scale is below 64,
  __shared__ int s_rec_Ec[OZ_MAXST][OZ_MAXA];   // the column scales of its chunk
  __shared__ int s_start[2];                    // tile (by parity) starts a chunk
  __shared__ __align__(8) uint64_t s_sfull[OZ_MAXST];
  __shared__ __align__(8) uint64_t s_sready[OZ_MAXST];
  __shared__ __align__(8) uint64_t s_sempty[OZ_MAXST];
  __shared__ __align__(8) uint64_t s_full[OZ_KS];
  __shared__ __align__(8) uint64_t s_empty[OZ_KS];
  __shared__ __align__(8) uint64_t s_tile[OZ_TRING];
  __shared__ __align__(8) uint64_t s_drained;
  __shared__ __align__(8) uint64_t s_final;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_code(P.status) != 0;
  __syncthreads();
  if (s_skip) return;

  const int a = rp.a, b = rp.b, nA = D.nA, N = D.N, nst = D.nst;
  unsigned char* Bs = smem + D.off_B;
  for (int t = tid; t < OZ_KS * N * 8; t += OZ_NT) reinterpret_cast<uint32_t*>(Bs)[t] = 0u;
  for (int t = tid; t < OZ_MAXA; t += OZ_NT) s_bad[t] = 0;
  if (tid == 0) {
    s_abort = 0;
    s_aborted = 0;
    s_issued = 0;
    s_landed = 0;
    s_start[0] = s_start[1] = 0;
    for (int s = 0; s < nst; ++s) {
      mbar_init(&s_sfull[s], 1);
      mbar_init(&s_sready[s], 1);
      mbar_init(&s_sempty[s], OZ_SPLIT / 32);
    }
    for (int s = 0; s < OZ_KS; ++s) {
      mbar_init(&s_full[s], 4);
      mbar_init(&s_empty[s], 1);
    }
    for (int s = 0; s < OZ_TRING; ++s) mbar_init(&s_tile[s], 1);
    mbar_init(&s_drained, OZ_SPLIT / 32);
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
  const uint32_t tA = s_tmem;               // A: K-step slot s at columns 32 s, region q at + 8 q
  const uint32_t tD = s_tmem + 32 * OZ_KS;  // D_q at columns 256 + q N
  const int first = blockIdx.x;
  const int ntl = first < P.ntiles ? (P.ntiles - first + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  // a column's 16-row piece of K-step ks in a stage: X columns first, then Y columns
  auto colrow = [&](const unsigned char* sb, int c, int ks) -> const unsigned char* {
    return c < a ? sb + ks * D.xbox + c * 128 : sb + OZ_KS * D.xbox + ks * D.ybox + (c - a) * 128;
  };

  if (warp == OZ_TMA_WARP) {
    // ======================= tensor copies of the row tiles ================================
    if (lane == 0) {
      const uint32_t bytes = 1024u * (uint32_t)(a + b);  // 8 boxes of 16 rows per operand
      for (int it = 0; it < ntl; ++it) {
        const int st = it % nst;
        if (it >= nst && !wait_or_abort(&s_sempty[st], (uint32_t)(((it / nst) - 1) & 1), &s_abort)) {
          set_error(P.status, RBO_ERR_TIMEOUT, 16);
          break;
        }
        unsigned char* sb = smem + (size_t)st * D.stage_bytes;
        const int r0 = (first + it * (int)gridDim.x) * OZ_T;
        mbar_arrive_expect_tx(&s_sfull[st], bytes);
        for (int ks = 0; ks < OZ_KS; ++ks) {
          if (a > 0) tma_load_2d(sb + ks * D.xbox, &D.tmX, r0 + 16 * ks, &s_sfull[st]);
          tma_load_2d(sb + OZ_KS * D.xbox + ks * D.ybox, &D.tmY, r0 + 16 * ks, &s_sfull[st]);
        }
        s_issued = it + 1;
      }
    }
  } else if (warp == OZ_SCAN_WARP) {
    // ======================= exponent maxima and chunk decisions ===========================
    // lane l owns the columns l and l + 32; its chunk scales stay in registers
    int Ecl[2] = {0, 0};
    bool open = false;
    int tic = 0;
    for (int it = 0; it < ntl; ++it) {
      const int st = it % nst;
      const bool ok = __all_sync(0xffffffffu, wait_or_abort(&s_sfull[st], (uint32_t)((it / nst) & 1), &s_abort));
      if (!ok) {
        if (lane == 0) set_error(P.status, RBO_ERR_TIMEOUT, 11);
        break;
      }
      if (lane == 0) s_landed = it + 1;
      const unsigned char* sb = smem + (size_t)st * D.stage_bytes;
      int et[2];
      bool exceed = false;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        uint32_t m = 0;
        if (c < nA) {
          const int sw = (c < a ? c : c - a) & 7;
#pragma unroll
          for (int ks = 0; ks < OZ_KS; ++ks) {
            const unsigned char* rowp = colrow(sb, c, ks);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const uint4 u = *reinterpret_cast<const uint4*>(rowp + ((j ^ sw) << 4));
              m = max(m, max(u.y & 0x7FFFFFFFu, u.w & 0x7FFFFFFFu));
            }
          }
        }
        et[h] = (int)(m >> 20);
        // larger values would overflow the chunk's fixed point, much smaller ones would
        // lose bits (a column of zeros fits every window)
        if (c < nA) exceed |= et[h] > Ecl[h] || (et[h] != 0 && et[h] < Ecl[h] - OZ_WIN);
      }
      const bool newc = __any_sync(0xffffffffu, exceed) || !open || tic == OZ_CHUNK;
      if (newc) {
        Ecl[0] = et[0] + OZ_HEAD;
        Ecl[1] = et[1] + OZ_HEAD;
        open = true;
        tic = 0;
      }
      ++tic;
      bool careful = false;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        if (c < nA) {
          s_rec_Ec[st][c] = Ecl[h];
          if (et[h] == 0x7FF) s_bad[c] = 1;
          careful |= Ecl[h] < 64;
        }
      }
      careful = __any_sync(0xffffffffu, careful);
      if (lane == 0) {
        s_rec_newc[st] = newc ? 1 : 0;
        s_rec_careful[st] = careful ? 1 : 0;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&s_sready[st]);
    }
  } else if (warp == OZ_MMA_WARP) {
    // ======================= tensor-core products (one thread) =============================
    if (lane == 0) {
      const uint32_t id = idesc_f16(128, N);
      bool ok = true;
      int nchunk = 0;
      for (int it = 0; it < ntl && ok; ++it) {
        for (int ks = 0; ks < OZ_KS; ++ks) {
          if (!wait_or_abort(&s_full[ks], (uint32_t)(it & 1), &s_abort)) {
            set_error(P.status, RBO_ERR_TIMEOUT, 13);
            ok = false;
            break;
          }
          tc_fence_after();
          uint32_t acc = 1u;
          if (ks == 0 && *reinterpret_cast<volatile int*>(&s_start[it & 1])) {
            // a new chunk: its first products overwrite the accumulators once the
            // splitters have drained the previous chunk
            acc = 0u;
            if (nchunk > 0) {
              if (!wait_or_abort(&s_drained, (uint32_t)((nchunk - 1) & 1), &s_abort)) {
                set_error(P.status, RBO_ERR_TIMEOUT, 17);
                ok = false;
                break;
              }
              tc_fence_after();
            }
            ++nchunk;
          }
          const uint64_t db = smem_desc(smem_u32(Bs + (size_t)ks * N * 32), 128, 256);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            mma_f16(tD + (uint32_t)(q * N), tA + (uint32_t)(32 * ks + 8 * q), db, id, acc);
          mma_commit(&s_empty[ks]);
        }
        if (ok) mma_commit(&s_tile[it % OZ_TRING]);
      }
      // every product issued has completed before the tensor memory is freed
      mma_commit(&s_final);
      mbar_wait_bounded(&s_final, 0u);
    }
  } else {
    // ======================= splitters (warps 0-7) =========================================
    const int wg = warp >> 2, wq = warp & 3;
    const int p = lane & 1, cw = lane >> 1;
    // lane (c, p) of tensor-memory lane 32 wq + lane: columns 8 wq .. 8 wq + 7 and
    // 32 + 8 wq .. 32 + 8 wq + 7 in quarter wq (every c mod 8 in each warp: the swizzled
    // stage reads are free of bank conflicts, and narrow panels spread over the warps)
    const int c = 8 * (4 * (cw >> 3) + wq) + (cw & 7);
    const bool active = c < nA;
    const bool isY = active && c >= a;
    const int sw = (c < a ? c : c - a) & 7;  // the column's 128-byte swizzle row
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
    // Packed words of a row for parity p: U = [byte of digit p, 0x64, byte of digit
    // 2 + p, 0x64], V = [byte of digit 4 + p, 0x64, byte of digit 6 + p, 0x64] from
    // G = (low word: bytes 0-3, high word: bytes 4-7; digit I is byte 6 - I, byte 7 is
    // 0x64); for p = 1 the last byte of V is a placeholder (there is no digit 7).
    const uint32_t selU = p ? 0x7375u : 0x7476u, selV = p ? 0x7071u : 0x7072u;
    const uint32_t selUo = p ? 0x7476u : 0x7375u, selVo = p ? 0x7072u : 0x7071u;

    __int128 acc[OZ_MAXB];
    int ea[OZ_MAXB];
#pragma unroll
    for (int y = 0; y < OZ_MAXB; ++y) {
      acc[y] = 0;
      ea[y] = -1;
    }
    int Ec = 64;          // this column's scale in the open chunk (64: a zero column)
    int eY[OZ_MAXB];      // the Y columns' scales in the open chunk
#pragma unroll
    for (int y = 0; y < OZ_MAXB; ++y) eY[y] = 0;
    // drain D (every product of the chunk complete) into the 128-bit accumulators
    auto drain = [&]() {
      long long hi[OZ_MAXB], lo[OZ_MAXB];
#pragma unroll
      for (int y = 0; y < OZ_MAXB; ++y) {
        hi[y] = 0;
        lo[y] = 0;
      }
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const int q = 2 * wg + qq;
        const int I = 2 * q + p;
#pragma unroll
        for (int y = 0; y < OZ_MAXB; ++y) {
          if (y < b) {  // b is uniform: the loads stay warp-converged
            float v[8];
            tmem_ld8(tD + (uint32_t)(q * N + 8 * y) + lane_base, v);
            if (active && I <= 6) {
#pragma unroll
              for (int J = 0; J < 7; ++J) {
                const int Lv = I + J;
                if (Lv <= 7) {
                  const long long iv = (long long)__float2int_rn(v[J]);
                  if (Lv <= 3) hi[y] += iv << (8 * (3 - Lv));
                  else lo[y] += iv << (8 * (7 - Lv));
                }
              }
            }
          }
        }
      }
      if (active) {
#pragma unroll
        for (int y = 0; y < OZ_MAXB; ++y) {
          if (y < b) {
            const __int128 S = ((__int128)hi[y] << 32) + (__int128)lo[y];
            if (S != 0) {
              const int Tt = Ec + eY[y];
              if (ea[y] < 0) ea[y] = Tt;
              int sh = Tt - ea[y];
              // |S| < 2^81; a shift of at most 20 keeps the sum of the CTA's chunks far
              // below 2^127
              if (sh > 20) {
                acc[y] >>= (sh - 20);
                ea[y] += sh - 20;
                sh = 20;
              }
              if (sh >= 0) acc[y] += S << sh;
              else if (sh > -120) acc[y] += S >> (-sh);
            }
          }
        }
      }
    };

    bool open = false, fail = false;
    for (int it = 0; it < ntl && !fail; ++it) {
      const int st = it % nst;
      if (!__all_sync(0xffffffffu, wait_or_abort(&s_sready[st], (uint32_t)((it / nst) & 1), &s_abort))) {
        if (lane == 0) set_error(P.status, RBO_ERR_TIMEOUT, 12);
        fail = true;
        break;
      }
      const bool newc = s_rec_newc[st] != 0;
      const bool careful = s_rec_careful[st] != 0;
      if (newc) {
        if (open) {
          const int pt = it - 1;
          if (!__all_sync(0xffffffffu, wait_or_abort(&s_tile[pt % OZ_TRING], (uint32_t)((pt / OZ_TRING) & 1), &s_abort))) {
            if (lane == 0) set_error(P.status, RBO_ERR_TIMEOUT, 14);
            fail = true;
            break;
          }
          tc_fence_after();
          drain();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&s_drained);
        }
        Ec = active ? s_rec_Ec[st][c] : 64;
#pragma unroll
        for (int y = 0; y < OZ_MAXB; ++y) eY[y] = y < b ? s_rec_Ec[st][a + y] : 0;
        open = true;
      }
      if (tid == 0) s_start[it & 1] = newc ? 1 : 0;  // read with the K-step 0 of this tile
      const unsigned char* sb = smem + (size_t)st * D.stage_bytes;

      // ---- digits of this warpgroup's K-steps -----------------------------------------
#pragma unroll 1
      for (int kk = 0; kk < OZ_KPW; ++kk) {
        const int ks = wg + 2 * kk;
        // this thread's 8 values: rows 8 p .. 8 p + 7 of the K-step
        uint32_t vl[8], vh[8];
        if (active) {
          const unsigned char* rowp = colrow(sb, c, ks);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint4 u = *reinterpret_cast<const uint4*>(rowp + (((4 * p + i) ^ sw) << 4));
            vl[2 * i] = u.x;
            vh[2 * i] = u.y;
            vl[2 * i + 1] = u.z;
            vh[2 * i + 1] = u.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) vl[j] = vh[j] = 0u;
        }
        if (kk == OZ_KPW - 1) {
          __syncwarp();
          if (lane == 0) mbar_arrive(&s_sempty[st]);  // the stage may be refilled
        }
        uint32_t Us[8], Vs[8], Uo[8], Vo[8];
        if (careful) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            uint32_t gl, gh;
            oz_fix<true>(vl[j], vh[j], Ec, gl, gh);
            Us[j] = __byte_perm(gl, gh, selU);
            Vs[j] = __byte_perm(gl, gh, selV);
            Uo[j] = __byte_perm(gl, gh, selUo);
            Vo[j] = __byte_perm(gl, gh, selVo);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            uint32_t gl, gh;
            oz_fix<false>(vl[j], vh[j], Ec, gl, gh);
            Us[j] = __byte_perm(gl, gh, selU);
            Vs[j] = __byte_perm(gl, gh, selV);
            Uo[j] = __byte_perm(gl, gh, selUo);
            Vo[j] = __byte_perm(gl, gh, selVo);
          }
        }
        // the other half of the column, packed for this lane's parity
        uint32_t Ur[8], Vr[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          Ur[j] = __shfl_xor_sync(0xffffffffu, Uo[j], 1);
          Vr[j] = __shfl_xor_sync(0xffffffffu, Vo[j], 1);
        }
        // rows 0-7 come from the p = 0 lane, rows 8-15 from the p = 1 lane
        uint32_t U[16], V[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          U[j] = p ? Ur[j] : Us[j];
          V[j] = p ? Vr[j] : Vs[j];
          U[8 + j] = p ? Us[j] : Ur[j];
          V[8 + j] = p ? Vs[j] : Vr[j];
        }
        uint32_t w[32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          w[j] = oz_digits(U[2 * j], U[2 * j + 1], 0x5410u);       // digit p
          w[8 + j] = oz_digits(U[2 * j], U[2 * j + 1], 0x7632u);   // digit 2 + p
          w[16 + j] = oz_digits(V[2 * j], V[2 * j + 1], 0x5410u);  // digit 4 + p
          w[24 + j] = oz_digits(V[2 * j], V[2 * j + 1], 0x7632u);  // digit 6 (p = 0)
        }
        // the slot's previous products have completed (A and B may be overwritten)
        if (it > 0 && !__all_sync(0xffffffffu, wait_or_abort(&s_empty[ks], (uint32_t)((it - 1) & 1), &s_abort))) {
          if (lane == 0) set_error(P.status, RBO_ERR_TIMEOUT, 15);
          fail = true;
          break;
        }
        tc_fence_after();
        tmem_st32(tA + (uint32_t)(32 * ks) + lane_base, w);
        if (isY) {
          // B rows 8 yc + J (J = 2q + p), K halves 128 bytes apart; J = 7 (q = 3, p = 1)
          // is never read back
          unsigned char* Bk = Bs + (size_t)ks * N * 32 + (c - a) * 256;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int J = 2 * q + p;
            *reinterpret_cast<uint4*>(Bk + J * 16) = make_uint4(w[8 * q], w[8 * q + 1], w[8 * q + 2], w[8 * q + 3]);
            *reinterpret_cast<uint4*>(Bk + 128 + J * 16) =
                make_uint4(w[8 * q + 4], w[8 * q + 5], w[8 * q + 6], w[8 * q + 7]);
          }
          fence_proxy_async();  // B written through the generic proxy
        }
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_full[ks]);
      }
    }
    // ---- the last chunk ------------------------------------------------------------------
    if (!fail && open) {
      const int pt = ntl - 1;
      if (!__all_sync(0xffffffffu, wait_or_abort(&s_tile[pt % OZ_TRING], (uint32_t)((pt / OZ_TRING) & 1), &s_abort))) {
        if (lane == 0) set_error(P.status, RBO_ERR_TIMEOUT, 14);
        fail = true;
      } else {
        tc_fence_after();
        drain();
      }
    }
    if (fail) s_abort = 1;
    bar_split();  // every splitter is done with the stages: they hold the partials now
    if (!s_abort && active) {
      // per-CTA contributions of this thread's (warpgroup, digit parity): slot 2 wg + p
      double* comb = reinterpret_cast<double*>(smem);  // 4 x 64 x 8
#pragma unroll
      for (int y = 0; y < OZ_MAXB; ++y) {
        if (y < b)
          comb[((size_t)(2 * wg + p) * OZ_MAXA + c) * OZ_MAXB + y] =
              ea[y] >= 0 ? ldexp((double)acc[y], ea[y] - 2110) : 0.0;
      }
    }
  }
  // ---- free the tensor memory (every issued product has completed) -------------------------
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    // tensor copies issued past the last tile the scanner saw land (an aborted call)
    // land before the CTA exits
    const int issued = s_issued;
    for (int t = s_landed; t < issued; ++t)
      mbar_wait_bounded(&s_sfull[t % nst], (uint32_t)((t / nst) & 1));
    if (s_abort || read_code(P.status) != 0) s_aborted = 1;
  }
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem),
                 "r"(OZ_TMEM_COLS));
  }
  __syncthreads();
  if (s_aborted || P.L == 0) return;

  const double* comb = reinterpret_cast<const double*>(smem);
  double* mypart = P.partials + (size_t)blockIdx.x * P.L;
  for (int o = tid; o < P.no; o += OZ_NT) {
    const int i = o / b, y = o % b;
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) sum += comb[((size_t)k * OZ_MAXA + i) * OZ_MAXB + y];
    if (s_bad[i] || s_bad[a + y]) sum = __longlong_as_double(0x7FF8000000000000LL);
    mypart[o] = sum;
  }
  tree_reduce_epilogue(P, smem, &s_flag, &s_last);
}

std::mutex g_oz_mu;
int g_oz_smem_set[64] = {};

}  // namespace

// 2-D tensor map of a column-major float64 array (n rows, cols columns, leading
// dimension ld): boxes of 16 rows x cols columns with the 128-byte swizzle, out-of-range
// rows read as zero.
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
  const cuuint32_t box[2] = {16u, (cuuint32_t)cols};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims,
                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? RBO_OK : RBO_ERR_CUDA;
}

bool ozaki_gram_supported(const RowPass& rp) {
  if (!rp.ozaki || rp.C || rp.Tri || rp.write_y || rp.sk_d > 0 || rp.sk_gd > 0 || rp.sk_cg > 0 ||
      rp.mixed || rp.df64)
    return false;
  if (!rp.acc_x && !rp.acc_y) return false;
  if (rp.b < 1 || rp.b > OZ_MAXB) return false;
  const int a = rp.acc_x ? rp.a : 0;
  if (a < 0 || rp.n <= 0 || rp.n >= (int64_t)1 << 31) return false;
  // tensor copies: 16-byte aligned bases and column strides
  if (((uintptr_t)rp.Y & 15) != 0 || (rp.ldy % 2) != 0) return false;
  if (a > 0 && (((uintptr_t)rp.X & 15) != 0 || (rp.ldx % 2) != 0)) return false;
  return a + rp.b <= OZ_MAXA;
}

// Measured on GB300 (n = 1e6, b = 5): this kernel takes 0.30-0.34 ms whatever the width,
// the float64 pass 0.11 ms at a = 5, 0.33 ms at a = 30 and 0.56 ms at a = 56.
bool ozaki_gram_pays(const RowPass& rp) {
  const int a = rp.acc_x ? rp.a : 0;
  return a + rp.b >= 36;
}

int ozaki_gram_launch(const RowPass& rpin, Arena* ar, cudaStream_t st, int* launches, int num_sms) {
  RowPass rp = rpin;
  if (!rp.acc_x) { rp.a = 0; rp.X = nullptr; }
  if (!ozaki_gram_supported(rp)) return RBO_ERR_ARG;
  const int a = rp.a, b = rp.b;
  const int nA = a + b;
  const int N = ((8 * b + 15) / 16) * 16;
  const int zr = a + (rp.acc_y ? b : 0), no = zr * b, L = no;
  const int xbox = ((a + 7) / 8) * 1024, ybox = ((b + 7) / 8) * 1024;
  const int stage_bytes = OZ_KS * (xbox + ybox);
  const size_t budget = 168 * 1024;
  const int nst = (int)std::max<size_t>(2, std::min<size_t>(OZ_MAXST, budget / stage_bytes));
  size_t o = (size_t)nst * stage_bytes;
  const size_t off_B = o;
  o += (size_t)OZ_KS * N * 32;
  const size_t epi = 64 + ((size_t)L + 2) * 8 + (size_t)b * b * 2 * 8 + 64 * 8;
  const size_t comb = (size_t)4 * OZ_MAXA * OZ_MAXB * 8;
  size_t smem = std::max(o, std::max(epi, comb)) + 1024;  // + alignment slack of the base
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
  P.TP = OZ_T;
  P.ntiles = ntiles;
  P.use_bulk = 1;
  P.zr = zr;
  P.no = no;
  P.L = L;
  P.ngroups = ngroups;
  P.status = ar->status;
  P.off_red = 64;
  const size_t need = ((size_t)G * L + (size_t)ngroups * L) * 8;
  if (ar->red == nullptr || need > ar->red_bytes) return RBO_ERR_NOMEM;
  if (ngroups + 1 > ar->n_tickets) return RBO_ERR_NOMEM;
  P.partials = ar->red;
  P.gpart = ar->red + (size_t)G * L;
  P.tickets = ar->tickets;
  D.nA = nA;
  D.zr = zr;
  D.N = N;
  D.nst = nst;
  D.xbox = xbox;
  D.ybox = ybox;
  D.stage_bytes = stage_bytes;
  D.off_B = (int)off_B;
  {
    int e = make_tensor_map(&D.tmY, rp.Y, rp.n, b, rp.ldy);
    if (e == RBO_OK && a > 0) e = make_tensor_map(&D.tmX, rp.X, rp.n, a, rp.ldx);
    if (e != RBO_OK) return e;
  }
  ProfToken tok = prof_start(st);
  ozaki_gram_kernel<<<G, OZ_NT, smem, st>>>(D);
  if (prof_on()) {
    const double nn = (double)rp.n, A = a, B = b;
    const double by = 8.0 * nn * (A + B);
    double fl = 0.0;
    if (rp.acc_x) fl += 2.0 * nn * A * B;
    if (rp.acc_y) fl += nn * B * (B + 1.0);
    prof_stop(tok, st, RBO_PROF_OZAKI, by, fl, rp.tag);
  }
  if (launches) ++*launches;
  return note_cuda(cudaGetLastError());
}

}  // namespace rbo

// Device helpers: PTX wrappers (mbarrier, bulk async copy), the SplitMix64 sketch
// hash, status reporting and warp/block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rbo_internal.cuh"

namespace rbo {

constexpr int NT = 256;            // threads per CTA of the row pass
constexpr int ZMAX = 16;           // largest zeta supported
constexpr int DMAX = 4096;         // largest sketch size d
constexpr long long WAIT_CYCLES = 4000000000LL;  // bounded waits: ~2 s at 2 GHz

// ---- status ---------------------------------------------------------------------
__device__ __forceinline__ void set_error(DevStatus* st, int code, int where) {
  if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
}
__device__ __forceinline__ void set_breakdown(DevStatus* st, int block, int column, int stage) {
  if (atomicCAS(&st->code, 0, RBO_ERR_CHOL_BREAKDOWN) == 0) {
    st->block = block;
    st->column = column;
    st->stage = stage;
  }
}
__device__ __forceinline__ int read_code(const DevStatus* st) {
  return *((volatile const int*)&st->code);
}

// ---- SplitMix64 sparse-sign sketch ---------------------------------------------------
// Output i (i >= 1) of the SplitMix64 stream seeded with `seed` is
// mix(seed + i * 0x9E3779B97F4A7C15) (Steele, Lea & Flood 2014); row r of the
// basis owns outputs 64 r + c + 1.  Index = ((h >> 32) * d) >> 32, sign from bit 0.
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Entries of sketch column `row`: zeta distinct indices in [0, d) in draw order,
// signs as +-1.  Returns false when 64 draws did not give zeta distinct indices.
__device__ __forceinline__ bool sketch_column(uint64_t seed, uint64_t row, int d, int zeta,
                                              int (&idx)[ZMAX], int (&neg)[ZMAX]) {
  int cnt = 0;
  const uint64_t base = seed + (row * 64ULL + 1ULL) * 0x9E3779B97F4A7C15ULL;
  for (int c = 0; c < 64 && cnt < zeta; ++c) {
    uint64_t h = splitmix_mix(base + (uint64_t)c * 0x9E3779B97F4A7C15ULL);
    int ix = (int)(((h >> 32) * (uint64_t)d) >> 32);
    bool dup = false;
#pragma unroll
    for (int t = 0; t < ZMAX; ++t)
      if (t < cnt && idx[t] == ix) dup = true;
    if (!dup) {
#pragma unroll
      for (int t = 0; t < ZMAX; ++t)
        if (t == cnt) {
          idx[t] = ix;
          neg[t] = (int)(h & 1ULL);
        }
      ++cnt;
    }
  }
  return cnt == zeta;
}

// ---- Gaussian entries: SplitMix64 + Box-Muller ---------------------------------------
// Entry (k, r) of a Gaussian map with d rows: output i = r d + k + 1 of the SplitMix64
// stream seeded with seed ^ GAUSS_SALT; m1 = top 24 bits, u1 = fl32(m1 + 1/2) 2^-24 in
// (0, 1), u2 = (bits 16..39) 2^-24; theta = sqrt(-2 ln u1) cos(2 pi u2) (Box and Muller
// 1958) in float32 arithmetic.
constexpr uint64_t GAUSS_SALT = 0x2545F4914F6CDD1DULL;
__device__ __forceinline__ float gauss_entry(uint64_t seed, uint64_t r, int k, int d) {
  const uint64_t h = splitmix_mix((seed ^ GAUSS_SALT) +
                                  (r * (uint64_t)d + (uint64_t)k + 1ULL) * 0x9E3779B97F4A7C15ULL);
  const float u1 = ((float)(uint32_t)(h >> 40) + 0.5f) * 0x1p-24f;
  const float u2 = (float)(uint32_t)((h >> 16) & 0xFFFFFFULL) * 0x1p-24f;
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// ---- fixed-point tile sums (integer ALU) ----------------------------------------------
// A column of a tile with largest exponent field E is summed exactly in int64 fixed
// point with unit 2^(E - 1023 - 54): every finite value converts with |v| < 2^55
// (round half away from zero below the unit; zero and subnormal values give 0), so
// sums of up to 128 values stay below 2^62.
__device__ __forceinline__ long long fix_from_double(double y, int E) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(y);
  const int e = (int)((u >> 52) & 0x7FF);
  if (e == 0) return 0;
  const unsigned long long M = (u & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
  const int sh = e - E + 2;  // <= 2
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
// s * 2^(E - 1023 - 54) rounded to a float64 (ties away from zero), integer ALU only
__device__ __forceinline__ double double_from_fix(long long s, int E) {
  if (s == 0) return 0.0;
  const unsigned long long neg = s < 0 ? 1ULL : 0ULL;
  const unsigned long long a = neg ? (unsigned long long)(-s) : (unsigned long long)s;
  const int nb = 64 - __clzll((long long)a);
  int ef = nb + E - 55;
  unsigned long long m;
  if (nb > 53) {
    const int k = nb - 53;
    m = (a + (1ULL << (k - 1))) >> k;
    if (m >> 53) {
      m >>= 1;
      ++ef;
    }
  } else {
    m = a << (53 - nb);
  }
  if (ef <= 0) return 0.0;
  if (ef >= 0x7FF) return __longlong_as_double((long long)((neg << 63) | 0x7FF0000000000000ULL));
  return __longlong_as_double((long long)((neg << 63) | ((unsigned long long)ef << 52) | (m & 0xFFFFFFFFFFFFFULL)));
}

// ---- float64 -> float32 by integer operations ----------------------------------------
// The f64->f32 conversion instruction runs on the float64 pipe of this GPU; this
// version uses integer ALU only: round to nearest on the 29 dropped mantissa bits
// (ties away from zero), values below the float32 normal range flush to zero and
// values above it saturate to infinity.
__device__ __forceinline__ float f64_to_f32_int(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  unsigned sign = hi & 0x80000000u;
  int e = (int)((hi >> 20) & 0x7FF) - 1023 + 127;
  unsigned mag;
  if (e <= 0) {
    mag = 0u;
  } else if (e >= 255) {
    mag = 0x7F800000u;
  } else {
    unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    mag = (((unsigned)e << 23) | mant) + ((lo >> 28) & 1u);
  }
  return __uint_as_float(sign | mag);
}

// ---- PTX: mbarrier + bulk async copy (TMA engine, non-tensor form) ----------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of `bar` with a bound; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

// ---- reductions ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Block-wide sum (fixed shuffle tree, deterministic); `scratch` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < (int)(blockDim.x >> 5) ? scratch[lane] : 0.0;
    r = warp_sum(r);
    if (lane == 0) scratch[0] = r;
  }
  __syncthreads();
  r = scratch[0];
  __syncthreads();
  return r;
}

}  // namespace rbo

namespace rbo {
// ---- float32-pair ("df64") arithmetic on the FP32 pipe -------------------------------
// A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)), about 48
// significant bits.  Error-free transformations: TwoSum (Knuth) and the FMA-based
// TwoProduct (Dekker's product with a fused multiply-add); see Joldes, Muller and
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 2017.
struct df {
  float h, l;
};

// float64 -> float pair with integer operations only: hi = the leading 24 bits
// (truncated), lo = the next 29 bits rounded to a float.  Values below 2^-74 in
// magnitude keep only hi (relative error 2^-24), values below the float32 normal
// range flush to zero.
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(u >> 32), lo32 = (unsigned)u;
  const unsigned sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7FF);   // biased float64 exponent
  const int ef = e - 1023 + 127;
  df r;
  if (ef <= 0 || e == 0x7FF) {
    if (e == 0x7FF) {  // inf / nan: propagate in hi
      r.h = __uint_as_float(sign | 0x7F800000u | (((hi32 & 0xFFFFFu) | lo32) ? 0x400000u : 0u));
    } else {
      r.h = 0.0f;
    }
    r.l = 0.0f;
    return r;
  }
  if (ef >= 255) {
    r.h = __uint_as_float(sign | 0x7F800000u);
    r.l = 0.0f;
    return r;
  }
  const unsigned mant23 = ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);
  r.h = __uint_as_float(sign | ((unsigned)ef << 23) | mant23);
  const unsigned rem = lo32 & 0x1FFFFFFFu;  // the 29 mantissa bits below hi
  // lo = rem * 2^(e - 1023 - 52): the float 2^(e-1023-52) has biased exponent ef - 52
  const int el = ef - 52;
  if (rem == 0u || el < 1) {
    r.l = 0.0f;
  } else {
    const float lo = __uint2float_rn(rem) * __uint_as_float((unsigned)el << 23);
    r.l = sign ? -lo : lo;
  }
  return r;
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // |a| >= |b|
  df r;
  r.h = a + b;
  r.l = b - (r.h - a);
  return r;
}

// acc += x * y  (all float pairs), accumulator not renormalised (l absorbs the errors)
__device__ __forceinline__ void df_fma_acc(df& acc, df x, df y) {
  const float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  const float s = acc.h + p;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) + (p - bb);
  acc.l += err + e;
  acc.h = s;
}

// acc += v (v a float pair)
__device__ __forceinline__ void df_add_acc(df& acc, df v) {
  const float s = acc.h + v.h;
  const float bb = s - acc.h;
  const float err = (acc.h - (s - bb)) + (v.h - bb);
  acc.l += err + v.l;
  acc.h = s;
}

__device__ __forceinline__ df df_norm(df a) { return df_fast_two_sum(a.h, a.l); }

// a * b (renormalised)
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.h, -a.l}; }
}  // namespace rbo

namespace rbo {
// float -> double by integer operations (exact; float subnormals flush to zero)
__device__ __forceinline__ double f32_to_f64_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  if (e == 0xFFu) return __hiloint2double((int)(sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u)), 0);
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}
// float pair -> double (one float64 addition)
__device__ __forceinline__ double df_to_double_fast(df a) {
  return f32_to_f64_int(a.h) + f32_to_f64_int(a.l);
}
}  // namespace rbo

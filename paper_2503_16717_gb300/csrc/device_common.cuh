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

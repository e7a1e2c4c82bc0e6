// Tensor-core message and node-update layers of the learned-SPAI network.
//
// Both layers apply a 64 -> 32 linear map with bfloat16 weights to one input vector per
// item, then the bias, a ReLU and a residual add:
//   message (per edge (i, j)):  m_ij = relu(Wm [e_ij ; h_j] + bm),  e_ij' = e_ij + m_ij
//   node update (per node i):   agg_i = sum_j m_ij,  r_i = relu(Wh [h_i ; agg_i] + bh),
//                               h_i' = h_i + r_i
// Over a tile of items the map is a dense contraction, Z (items x 32) = X (items x 64) W^T,
// done here by tcgen05.mma with M = 128 items, N = 32 outputs, K = 64 inputs.
//
// Precision.  X is float32.  Every value is split into three bfloat16 pieces,
// x = x0 + x1 + x2 + r with x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1) (each
// difference is exact in float32) and |r| <= 2^-27 |x|, below float32's own rounding.  A
// piece times a bfloat16 weight is exact in float32, so Z = [X0 X1 X2] [W W W]^T (K = 192)
// is X W^T to float32 accuracy, summed in the tensor core's float32 accumulator.
//
// Work of one CTA (128 threads, 4 warps; warp q owns tensor-memory lanes 32q..32q+31 =
// items 32q..32q+31 of the tile), per tile:
//   1. the warp loads its 32 items' inputs with lane = channel (coalesced 128-byte rows;
//      the node layer also sums each node's incoming messages, edges in CSR order) into
//      a per-warp buffer with row = item (stride 65 floats: the lane = channel writes and
//      the row-per-thread reads are both free of bank conflicts);
//   2. thread t reads row t, splits it and stores the pieces to tensor memory (A: piece p
//      at columns 32p..32p+31, two bfloat16 per 32-bit column in K order);
//   3. one thread issues the 12 MMAs (3 pieces x 4 K-steps of 16) into D (columns
//      96..127), B = W in shared memory (K-major, no swizzle), and commits to an mbarrier;
//   4. thread t loads row t of D into its buffer row, and the warp reads the outputs back
//      with lane = channel for the epilogue and coalesced stores.
// Four CTAs per SM (a quarter of tensor memory each) overlap one CTA's loads with
// another's products.  Every wait is bounded; a timeout sets RBO_ERR_TIMEOUT.
#include <cuda_bf16.h>

#include <algorithm>

#include "device_common.cuh"
#include "gnn_params.cuh"

namespace rbo {
namespace gnn {
namespace {

constexpr int TT = 128;               // items per tile (MMA M)
constexpr int TNT = 128;              // threads per CTA
constexpr int TLD = 65;               // row stride of the per-warp buffers (floats)
constexpr uint32_t TCOLS = 128;       // tensor-memory columns per CTA: A 96, D 32
constexpr uint32_t TD = 96;           // first column of D
constexpr int TCTAS = 4;              // CTAs per SM
constexpr int OFF_B = 4 * 32 * TLD * 4;  // B after the four warp buffers (33280 bytes)
constexpr int SMEM_USED = OFF_B + 4096;  // B: 4 K-steps x 32 rows x 32 bytes
// dynamic shared memory per CTA: the used part, alignment slack, and enough padding that
// at most four CTAs fit on an SM (each holds a quarter of the tensor memory)
constexpr int TSMEM = 47 * 1024;
static_assert(SMEM_USED + 1024 <= TSMEM, "tensor-core GNN layout exceeds its shared memory");

__device__ __forceinline__ float relu_tc(float x) { return x > 0.f ? x : 0.f; }

// no-swizzle canonical shared-memory descriptor: start, leading (K) byte offset, stride
// (M/N) byte offset, all >> 4; descriptor version 1 at bits 46-48
__device__ __forceinline__ uint64_t desc_nosw(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}
// kind::f16 instruction descriptor: D float32 (bits 4-5 = 1), A and B bfloat16 (bits 7-9
// and 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
// D (tensor memory) [+]= A (tensor memory) B (shared memory descriptor)
__device__ __forceinline__ void mma_bf16(uint32_t d, uint32_t a, uint64_t b, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
      "r"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit_to(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 32 consecutive 32-bit columns of this thread's lane; the wait is in the same statement
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

// B = W (32 outputs x 64 inputs, row-major bfloat16 at w + off), K-major no-swizzle core
// matrices: K-step k / 16 at 1024 bytes, 8-row group n / 8 at 256, K half (k % 16) / 8 at
// 128 (the leading byte offset), row n % 8 at 16, element k % 8 at 2
__device__ __forceinline__ void fill_weights(unsigned char* Bs, const __nv_bfloat16* __restrict__ w,
                                             int off) {
  for (int t = threadIdx.x; t < 32 * 64; t += blockDim.x) {
    const int n = t >> 6, k = t & 63;
    const int o = (k >> 4) * 1024 + (n >> 3) * 256 + ((k >> 3) & 1) * 128 + (n & 7) * 16 + (k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(Bs + o) = w[off + t];
  }
}

// Thread's row of 64 float32 inputs -> three bfloat16 pieces in its tensor-memory lane:
// piece p, inputs 32h..32h+31 at columns 32p + 16h .. +15
__device__ __forceinline__ void split_to_tmem(const float* row, uint32_t tlane) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float r[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) r[k] = row[32 * h + k];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      uint32_t wd[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(r[2 * j], r[2 * j + 1]);
        const float2 f = __bfloat1622float2(b);
        r[2 * j] -= f.x;  // exact: the remainder of a rounding to 8 significant bits
        r[2 * j + 1] -= f.y;
        wd[j] = *reinterpret_cast<const uint32_t*>(&b);
      }
      tmem_st16(tlane + (uint32_t)(32 * p + 16 * h), wd);
    }
  }
}

// Shared part of the two kernels: split the tile's inputs (the warp buffers, rows =
// items), run the products, and leave each item's 32 outputs in columns 32..63 of its
// buffer row.  false: the wait for the products timed out (for every thread of the CTA).
__device__ __forceinline__ bool tile_products(float* buf, uint32_t tbase, uint32_t tlane,
                                              const unsigned char* Bs, uint64_t* bar, int it) {
  const int lane = threadIdx.x & 31;
  split_to_tmem(buf + lane * TLD, tlane);
  tmem_st_wait();
  tc_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc_after();
    const uint32_t id = idesc_bf16(TT, 32);
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        mma_bf16(tbase + TD, tbase + (uint32_t)(32 * p + 8 * ks),
                 desc_nosw(smem_u32(Bs + ks * 1024), 128, 256), id, (p | ks) != 0 ? 1u : 0u);
    mma_commit_to(bar);
  }
  const bool ok = mbar_wait_bounded(bar, (uint32_t)(it & 1));
  if (__syncthreads_or(!ok)) return false;
  tc_after();
  uint32_t z[32];
  tmem_ld32(tlane + TD, z);
#pragma unroll
  for (int c = 0; c < 32; ++c) buf[lane * TLD + 32 + c] = __uint_as_float(z[c]);
  __syncwarp();
  return true;
}

// Set-up shared by the two kernels: weights into B, the mbarrier, tensor memory
__device__ __forceinline__ void tc_setup(unsigned char* Bs, const __nv_bfloat16* __restrict__ w,
                                         int off, uint64_t* bar, uint32_t* s_tmem) {
  fill_weights(Bs, w, off);
  fence_proxy_async();  // B written through the generic proxy, read by the tensor core
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(s_tmem)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before();
  __syncthreads();
  tc_after();
}

// Every product issued has completed before the tensor memory is freed
__device__ __forceinline__ void tc_teardown(uint64_t* fin, uint32_t tbase) {
  if (threadIdx.x == 0) {
    mma_commit_to(fin);
    mbar_wait_bounded(fin, 0u);
  }
  tc_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TCOLS));
  }
}

__device__ __forceinline__ unsigned char* align1k(unsigned char* p) {
  return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}

}  // namespace

// message layer l over all edges (see the file header); edge q = (row i, col[q] = j)
__global__ void __launch_bounds__(TNT, TCTAS)
    message_tc_kernel(int64_t nnz, int64_t n, const int32_t* __restrict__ col,
                      const float* __restrict__ ein, const float* __restrict__ h,
                      const __nv_bfloat16* __restrict__ w, int l, float* __restrict__ m,
                      float* __restrict__ eout, DevStatus* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mma, s_fin;
  __shared__ int s_skip;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_code(status) != 0;
  __syncthreads();
  if (s_skip) return;
  unsigned char* smem = align1k(smem_raw);
  float* buf = reinterpret_cast<float*>(smem) + warp * 32 * TLD;
  const unsigned char* Bs = smem + OFF_B;
  if (tid == 0) mbar_init(&s_fin, 1);
  tc_setup(smem + OFF_B, w, off_wm(l), &s_mma, &s_tmem);
  const uint32_t tbase = s_tmem;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
  const float bias = __bfloat162float(w[off_bm(l) + lane]);
  const int64_t ntiles = (nnz + TT - 1) / TT;
  bool bad = false;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t e0 = tile * TT + warp * 32;
    int cj = -1;
    if (e0 + lane < nnz) {
      cj = col[e0 + lane];
      if (cj < 0 || (int64_t)cj >= n) {
        bad = true;
        cj = -1;
      }
    }
    float ev[32], hv[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = __shfl_sync(0xffffffffu, cj, j);
      ev[j] = e0 + j < nnz ? ein[(e0 + j) * W + lane] : 0.f;
      hv[j] = c >= 0 ? h[(int64_t)c * W + lane] : 0.f;
    }
    __syncwarp();  // the previous tile's reads of the buffer are done
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      buf[j * TLD + lane] = ev[j];
      buf[j * TLD + 32 + lane] = hv[j];
    }
    __syncwarp();
    if (!tile_products(buf, tbase, tlane, Bs, &s_mma, it)) {
      if (tid == 0) set_error(status, RBO_ERR_TIMEOUT, 40);
      break;
    }
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      if (e0 + j < nnz) {
        const float mv = relu_tc(buf[j * TLD + 32 + lane] + bias);
        m[(e0 + j) * W + lane] = mv;
        eout[(e0 + j) * W + lane] = buf[j * TLD + lane] + mv;
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(status, RBO_ERR_ARG, 41);
  tc_teardown(&s_fin, tbase);
}

// aggregation + node update of layer l over all nodes (see the file header)
__global__ void __launch_bounds__(TNT, TCTAS)
    node_update_tc_kernel(int64_t n, const int32_t* __restrict__ rowptr, const float* __restrict__ m,
                          const float* __restrict__ hin, const __nv_bfloat16* __restrict__ w, int l,
                          float* __restrict__ agg, float* __restrict__ rh, float* __restrict__ hout,
                          DevStatus* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mma, s_fin;
  __shared__ int s_skip;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_code(status) != 0;
  __syncthreads();
  if (s_skip) return;
  unsigned char* smem = align1k(smem_raw);
  float* buf = reinterpret_cast<float*>(smem) + warp * 32 * TLD;
  const unsigned char* Bs = smem + OFF_B;
  if (tid == 0) mbar_init(&s_fin, 1);
  tc_setup(smem + OFF_B, w, off_wh(l), &s_mma, &s_tmem);
  const uint32_t tbase = s_tmem;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
  const float bias = __bfloat162float(w[off_bh(l) + lane]);
  const int64_t ntiles = (n + TT - 1) / TT;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t i0 = tile * TT + warp * 32;
    // row starts of the warp's 32 nodes (lanes past the last node: rowptr[n], above every
    // edge of the range) and the end of the warp's edge range
    const int rs = rowptr[std::min<int64_t>(i0 + lane, n)];
    const int E0 = __shfl_sync(0xffffffffu, rs, 0);
    const int E1 = rowptr[std::min<int64_t>(i0 + 32, n)];
    float hv[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) hv[j] = i0 + j < n ? hin[(i0 + j) * W + lane] : 0.f;
    __syncwarp();  // the previous tile's reads of the buffer are done
#pragma unroll
    for (int j = 0; j < 32; ++j) buf[j * TLD + 32 + lane] = 0.f;  // nodes without edges
    // incoming messages in CSR order, 16 edges in flight; an edge belongs to the last node
    // whose row starts at or before it; each node's sum starts from 0 and adds its edges
    // in order
    int cur = -1;
    float run = 0.f;
    for (int e = E0; e < E1; e += 16) {
      float v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = e + u < E1 ? m[(int64_t)(e + u) * W + lane] : 0.f;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        if (e + u < E1) {
          const unsigned mask = __ballot_sync(0xffffffffu, rs <= e + u);
          const int j = 31 - __clz((int)mask);
          if (j != cur) {
            if (cur >= 0) buf[cur * TLD + 32 + lane] = run;
            run = 0.f;
            cur = j;
          }
          run += v[u];
        }
      }
    }
    if (cur >= 0) buf[cur * TLD + 32 + lane] = run;
#pragma unroll
    for (int j = 0; j < 32; ++j) buf[j * TLD + lane] = hv[j];
    __syncwarp();
#pragma unroll 8
    for (int j = 0; j < 32; ++j)
      if (i0 + j < n) agg[(i0 + j) * W + lane] = buf[j * TLD + 32 + lane];
    __syncwarp();  // agg read before tile_products overwrites the columns with outputs
    if (!tile_products(buf, tbase, tlane, Bs, &s_mma, it)) {
      if (tid == 0) set_error(status, RBO_ERR_TIMEOUT, 42);
      break;
    }
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      if (i0 + j < n) {
        const float r = relu_tc(buf[j * TLD + 32 + lane] + bias);
        rh[(i0 + j) * W + lane] = r;
        hout[(i0 + j) * W + lane] = buf[j * TLD + lane] + r;
      }
    }
  }
  tc_teardown(&s_fin, tbase);
}

static int tc_grid(int64_t items) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (items + TT - 1) / TT;
  return (int)std::min<int64_t>(tiles, (int64_t)TCTAS * std::max(sms, 1));
}

int message_tc_launch(int64_t nnz, int64_t n, const int32_t* col, const float* ein, const float* h,
                      const __nv_bfloat16* w, int l, float* m, float* eout, DevStatus* status,
                      cudaStream_t st) {
  if (nnz <= 0) return RBO_OK;
  message_tc_kernel<<<tc_grid(nnz), TNT, TSMEM, st>>>(nnz, n, col, ein, h, w, l, m, eout, status);
  return note_cuda(cudaGetLastError());
}

int node_update_tc_launch(int64_t n, const int32_t* rowptr, const float* m, const float* hin,
                          const __nv_bfloat16* w, int l, float* agg, float* rh, float* hout,
                          DevStatus* status, cudaStream_t st) {
  if (n <= 0) return RBO_OK;
  node_update_tc_kernel<<<tc_grid(n), TNT, TSMEM, st>>>(n, rowptr, m, hin, w, l, agg, rh, hout,
                                                        status);
  return note_cuda(cudaGetLastError());
}

}  // namespace gnn
}  // namespace rbo

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
// x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1): each difference is exact in
// float32, and x = x0 + x1 + x2 exactly (x has 24 significant bits, the first remainder
// at most 16, the second at most 8, which bfloat16 holds).  A piece times a bfloat16
// weight is exact in float32, so Z = [X0 X1 X2] [W W W]^T (K = 192) is X W^T with only
// the float32 rounding of the tensor core's accumulator.
//
// Work of one CTA (128 threads, 4 warps; warp q owns tensor-memory lanes 32q..32q+31 =
// items 32q..32q+31 of the tile), per tile:
//   1. the warp loads its 32 items' inputs with lane = channel (coalesced 128-byte rows;
//      the node layer also sums each node's incoming messages, edges in CSR order, 32
//      message rows in flight per warp) into a per-warp buffer with row = item (stride
//      65 floats: the lane = channel writes and the row-per-thread reads are both free
//      of bank conflicts);
//   2. thread t reads row t, splits it and stores the pieces to tensor memory (A: piece p
//      at columns 32p..32p+31, two bfloat16 per 32-bit column in K order);
//   3. one thread issues the 12 MMAs (3 pieces x 4 K-steps of 16) into D (columns
//      96..127), B = W in shared memory (K-major, no swizzle), and commits to an mbarrier;
//   4. thread t loads row t of D into its buffer row, and the warp reads the outputs back
//      with lane = channel for the epilogue and coalesced stores.
// Four CTAs per SM (a quarter of tensor memory each) overlap one CTA's loads with
// another's products.  Every wait is bounded; a timeout sets RBO_ERR_TIMEOUT.
// In inference the first message layer computes e_0 from the edge features (the edge
// encoder) and the last message and node layers compute the decoder's dot products, so
// neither e_0 nor the last e and h need to be stored.  The backward of both layers (two
// more contractions per tile) follows the forward kernels below.
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
// 32 consecutive 32-bit columns of this thread's lane
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

// Arguments of a message layer.  The first layer takes the edge features x (3 per edge)
// instead of e_0 and computes e_0 = relu(We x + be) on the fly (the edge encoder); the
// last one can leave e_{l+1} unwritten and write the decoder's edge term instead.
struct MsgArgs {
  int64_t nnz, n;
  const int32_t* col;        // column j of edge q
  const float* ein;          // e_l per edge; null: e_0 from x
  const float* x;            // edge features, 3 per edge (used when ein is null)
  float* e0out;              // e_0 written here when computed and non-null
  const float* h;            // h_l per node (gathered by column)
  const __nv_bfloat16* w;    // bfloat16 parameters
  int l;                     // layer
  float* m;                  // m_l per edge
  float* eout;               // e_{l+1} = e_l + m_l per edge, or null
  float* pe;                 // decoder edge term wo[0:32] . e_{l+1} per edge, or null
  DevStatus* status;
};

// message layer l over all edges (see the file header); edge q = (row i, col[q] = j).
// ENC: e_0 from the edge features (first layer); PE: the decoder's edge term (last layer)
template <bool ENC, bool PE>
__global__ void __launch_bounds__(TNT, TCTAS) message_tc_kernel(const __grid_constant__ MsgArgs P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mma, s_fin;
  __shared__ int s_skip;
  __shared__ float s_bias[32], s_wo[32], s_we[96], s_be[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_code(P.status) != 0;
  __syncthreads();
  if (s_skip) return;
  unsigned char* smem = align1k(smem_raw);
  float* buf = reinterpret_cast<float*>(smem) + warp * 32 * TLD;
  const unsigned char* Bs = smem + OFF_B;
  if (tid == 0) mbar_init(&s_fin, 1);
  tc_setup(smem + OFF_B, P.w, off_wm(P.l), &s_mma, &s_tmem);
  const uint32_t tbase = s_tmem;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);
  const float bias = __bfloat162float(P.w[off_bm(P.l) + lane]);
  if (warp == 0) {  // layer bias, decoder edge weights, edge encoder (first layer)
    s_bias[lane] = bias;
    s_wo[lane] = __bfloat162float(P.w[OFF_WO + lane]);
    s_be[lane] = __bfloat162float(P.w[OFF_BE + lane]);
    for (int k = 0; k < 3; ++k) s_we[32 * k + lane] = __bfloat162float(P.w[OFF_WE + 32 * k + lane]);
  }
  __syncthreads();
  const int64_t nnz = P.nnz;
  const int64_t ntiles = (nnz + TT - 1) / TT;
  bool bad = false;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t e0 = tile * TT + warp * 32;
    int cj = -1;
    if (e0 + lane < nnz) {
      cj = P.col[e0 + lane];
      if (cj < 0 || (int64_t)cj >= P.n) {
        bad = true;
        cj = -1;
      }
    }
    float ev[32], hv[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = __shfl_sync(0xffffffffu, cj, j);
      if constexpr (!ENC) ev[j] = e0 + j < nnz ? P.ein[(e0 + j) * W + lane] : 0.f;
      hv[j] = c >= 0 ? P.h[(int64_t)c * W + lane] : 0.f;
    }
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;  // first layer: this thread's edge features
    if (ENC && e0 + lane < nnz) {
      x0 = P.x[3 * (e0 + lane)];
      x1 = P.x[3 * (e0 + lane) + 1];
      x2 = P.x[3 * (e0 + lane) + 2];
    }
    __syncwarp();  // the previous tile's reads of the buffer are done
    if constexpr (ENC) {
      // the edge encoder for this thread's edge, in the order of its own kernel (bias,
      // then inputs 0..2), into its buffer row
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        float z = s_be[c];
        z = fmaf(s_we[3 * c], x0, z);
        z = fmaf(s_we[3 * c + 1], x1, z);
        z = fmaf(s_we[3 * c + 2], x2, z);
        buf[lane * TLD + c] = e0 + lane < nnz ? relu_tc(z) : 0.f;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) buf[j * TLD + lane] = ev[j];
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) buf[j * TLD + 32 + lane] = hv[j];
    __syncwarp();
    if (ENC && P.e0out) {
#pragma unroll 8
      for (int j = 0; j < 32; ++j)
        if (e0 + j < nnz) P.e0out[(e0 + j) * W + lane] = buf[j * TLD + lane];
    }
    if (!tile_products(buf, tbase, tlane, Bs, &s_mma, it)) {
      if (tid == 0) set_error(P.status, RBO_ERR_TIMEOUT, 40);
      break;
    }
    if constexpr (PE) {  // this thread's edge: wo[0:32] . e_{l+1} from its buffer row
      float t = 0.f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float mv = relu_tc(buf[lane * TLD + 32 + c] + s_bias[c]);
        t = fmaf(s_wo[c], buf[lane * TLD + c] + mv, t);
      }
      if (e0 + lane < nnz) P.pe[e0 + lane] = t;
    }
    float* __restrict__ eout = P.eout;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      if (e0 + j < nnz) {
        const float mv = relu_tc(buf[j * TLD + 32 + lane] + bias);
        P.m[(e0 + j) * W + lane] = mv;
        if (eout) eout[(e0 + j) * W + lane] = buf[j * TLD + lane] + mv;
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(P.status, RBO_ERR_ARG, 41);
  tc_teardown(&s_fin, tbase);
}

// aggregation + node update of layer l over all nodes (see the file header)
// agg, rh and hout may be null (inference keeps only what the next layer reads); sdec
// and tdec, when non-null, receive the decoder's node terms wo[32:64] . h' and
// wo[64:96] . h' (the last layer)
__global__ void __launch_bounds__(TNT, TCTAS)
    node_update_tc_kernel(int64_t n, const int32_t* __restrict__ rowptr, const float* __restrict__ m,
                          const float* __restrict__ hin, const __nv_bfloat16* __restrict__ w, int l,
                          float* __restrict__ agg, float* __restrict__ rh, float* __restrict__ hout,
                          float* __restrict__ sdec, float* __restrict__ tdec, DevStatus* status) {
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
  __shared__ float s_bias[32], s_woi[32], s_woj[32];
  if (warp == 0) {  // read after the first tile's barriers
    s_bias[lane] = bias;
    s_woi[lane] = __bfloat162float(w[OFF_WO + W + lane]);
    s_woj[lane] = __bfloat162float(w[OFF_WO + 2 * W + lane]);
  }
  __syncthreads();
  const int64_t ntiles = (n + TT - 1) / TT;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t i0 = tile * TT + warp * 32;
    // row starts of the warp's 32 nodes (lanes past the last node: rowptr[n], above every
    // edge of the range) and the end of the warp's edge range
    const int rs = rowptr[std::min<int64_t>(i0 + lane, n)];
    const int E0 = __shfl_sync(0xffffffffu, rs, 0);
    const int E1 = rowptr[std::min<int64_t>(i0 + 32, n)];
    {
      float hv[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) hv[j] = i0 + j < n ? hin[(i0 + j) * W + lane] : 0.f;
      __syncwarp();  // the previous tile's reads of the buffer are done
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        buf[j * TLD + lane] = hv[j];
        buf[j * TLD + 32 + lane] = 0.f;  // nodes without edges
      }
    }
    // incoming messages in CSR order, 32 edges in flight; an edge belongs to the last node
    // whose row starts at or before it; each node's sum starts from 0 and adds its edges
    // in order
    int cur = -1;
    float run = 0.f;
    for (int e = E0; e < E1; e += 32) {
      float v[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) v[u] = e + u < E1 ? m[(int64_t)(e + u) * W + lane] : 0.f;
#pragma unroll
      for (int u = 0; u < 32; ++u) {
        // branch-free: a new node stores the previous node's sum and restarts from this
        // edge (0 + v = v, the same value as an explicit restart); edges past the range
        // keep the node and add 0
        const unsigned mask = __ballot_sync(0xffffffffu, rs <= e + u);
        const int j = e + u < E1 ? 31 - __clz((int)mask) : cur;
        const bool fresh = j != cur;
        if (fresh && cur >= 0) buf[cur * TLD + 32 + lane] = run;
        run = fresh ? v[u] : run + v[u];
        cur = j;
      }
    }
    if (cur >= 0) buf[cur * TLD + 32 + lane] = run;
    __syncwarp();
    if (agg) {
#pragma unroll 8
      for (int j = 0; j < 32; ++j)
        if (i0 + j < n) agg[(i0 + j) * W + lane] = buf[j * TLD + 32 + lane];
    }
    __syncwarp();  // agg read before tile_products overwrites the columns with outputs
    if (!tile_products(buf, tbase, tlane, Bs, &s_mma, it)) {
      if (tid == 0) set_error(status, RBO_ERR_TIMEOUT, 42);
      break;
    }
    if (sdec) {  // this thread's node: wo[32:64] . h' and wo[64:96] . h' from its buffer row
      float si = 0.f, tj = 0.f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float hn = buf[lane * TLD + c] + relu_tc(buf[lane * TLD + 32 + c] + s_bias[c]);
        si = fmaf(s_woi[c], hn, si);
        tj = fmaf(s_woj[c], hn, tj);
      }
      if (i0 + lane < n) {
        sdec[i0 + lane] = si;
        tdec[i0 + lane] = tj;
      }
    }
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {
      if (i0 + j < n) {
        const float r = relu_tc(buf[j * TLD + 32 + lane] + bias);
        if (rh) rh[(i0 + j) * W + lane] = r;
        if (hout) hout[(i0 + j) * W + lane] = buf[j * TLD + lane] + r;
      }
    }
  }
  tc_teardown(&s_fin, tbase);
}

// ---- backward of the message and node-update layers ------------------------------------
// Per item (edge q = (i, j) for the message layer, node i for the node update), with
// u = the layer's 64 inputs and a = its output after the ReLU:
//   dz = g * [a > 0]   (g = de_q + dagg_i for a message, dh_i for a node update)
//   dW += dz u^T,  db += dz,  du = W^T dz
//   outputs: g + du[0:32] (gradient of e_q or h_i), du[32:64] (of h_j per edge, or agg_i)
// Both contractions run on the tensor cores, per tile of 128 items:
//   du (M = 128 items, N = 64, K = 32): A = dz split into three bfloat16 pieces (tensor
//     memory, row = item), B = W^T (shared memory);
//   dW^T (M = 128 = (piece p of u, input k), N = 64 = (piece q of dz, output c), K = the
//     tile's items): A = the hi (p = 0) and lo (p = 1) bfloat16 pieces of u, row (p, k),
//     two items per 32-bit column; B = the hi and lo pieces of dz (shared memory, K = item);
//     accumulated in tensor memory over all tiles of the CTA.  The hi/lo split leaves a
//     remainder below 2^-16 of each value, so the four piece products sum to u dz^T
//     within 2^-15 relative per term.
// At the end each CTA writes its partial of dW (element (c, k) at k * 32 + c) and db
// (at 64 * 32 + c), summed over the CTAs in a fixed order by the reduction kernel.
struct BackArgs {
  int64_t cnt;               // items: edges or nodes
  int64_t n;                 // nodes (bound of the gathered indices)
  const int32_t* erow;       // message: row i of edge q
  const int32_t* col;        // message: column j of edge q
  const float* g;            // gradient reaching the item's output (de or dh), per item
  const float* dagg;         // message: gradient of each node's aggregate, added to de
  const float* act;          // the layer's output after the ReLU (m or rh), per item
  const float* u0;           // inputs 0..31 (e_l per edge, h_l per node), per item
  const float* u1;           // inputs 32..63 (h_l[j] gathered per edge, agg_l per node)
  const __nv_bfloat16* w;    // bfloat16 parameters
  int off_w;                 // the layer's 32 x 64 weight matrix
  float* out0;               // g + du[0:32]
  float* out1;               // du[32:64]
  float* part;               // per-CTA partials, 65 * 32 floats each
  DevStatus* status;
};

constexpr int BLD = 97;                         // buffer row: dz (32) | u (64), + 1
constexpr int BOFF_BDU = 49 * 1024;             // after 4 x 32 x 97 floats (49664 bytes)
constexpr int BOFF_BG = BOFF_BDU + 4096;        // B of du: 2 K-steps x 64 rows x 32 bytes
constexpr int BSMEM_USED = BOFF_BG + 16384;     // B of dW: 8 K-steps x 64 rows x 32 bytes
// dynamic shared memory per CTA: enough padding that at most two CTAs fit on an SM (each
// holds half of the tensor memory)
constexpr int BSMEM = 80 * 1024;
constexpr uint32_t BCOLS = 256;                 // tensor memory: A_du, D_du, A_dW, D_dW
constexpr uint32_t B_ADU = 0, B_DDU = 64, B_AG = 128, B_DG = 192;
static_assert(4 * 32 * BLD * 4 <= BOFF_BDU, "backward buffers overlap B");
static_assert(BSMEM_USED + 1024 <= BSMEM, "tensor-core GNN backward exceeds its shared memory");

template <bool MSG>
__global__ void __launch_bounds__(TNT, 2) layer_back_tc_kernel(const __grid_constant__ BackArgs P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mma, s_fin;
  __shared__ int s_skip;
  __shared__ float s_db[4][32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_skip = read_code(P.status) != 0;
  __syncthreads();
  if (s_skip) return;
  unsigned char* smem = align1k(smem_raw);
  float* bufs = reinterpret_cast<float*>(smem);
  float* buf = bufs + warp * 32 * BLD;
  unsigned char* Bdu = smem + BOFF_BDU;
  unsigned char* Bg = smem + BOFF_BG;
  // B of du = W^T: row n = input k, K index = output c (W[c][k] at w + off_w + 64 c + k)
  for (int t = tid; t < 32 * 64; t += TNT) {
    const int c = t >> 6, k = t & 63;
    const int o = (c >> 4) * 2048 + (k >> 3) * 256 + ((c >> 3) & 1) * 128 + (k & 7) * 16 + (c & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(Bdu + o) = P.w[P.off_w + t];
  }
  fence_proxy_async();
  if (tid == 0) {
    mbar_init(&s_mma, 1);
    mbar_init(&s_fin, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(BCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tb = s_tmem;
  const uint32_t tl = tb + ((uint32_t)(warp * 32) << 16);
  // this thread's row of the dW^T product: piece gp of input gk
  const int gk = 32 * (warp & 1) + lane, gp = warp >> 1;
  float db = 0.f;
  const int64_t ntiles = (P.cnt + TT - 1) / TT;
  bool bad = false, ok = true;
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int64_t q0 = tile * TT + warp * 32;
    int ri = -1, cj = -1;
    if (MSG && q0 + lane < P.cnt) {
      ri = P.erow[q0 + lane];
      cj = P.col[q0 + lane];
      if (ri < 0 || (int64_t)ri >= P.n || cj < 0 || (int64_t)cj >= P.n) {
        bad = true;
        ri = cj = -1;
      }
    }
    float r[32];
    __syncwarp();  // the previous tile's reads of the buffer are done
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float dz[16];
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = 16 * half + jj;
        const int64_t q = q0 + j;
        float gv = 0.f, av = 0.f, x0 = 0.f, x1 = 0.f;
        if (MSG) {
          const int i = __shfl_sync(0xffffffffu, ri, j);
          const int c = __shfl_sync(0xffffffffu, cj, j);
          if (q < P.cnt && i >= 0) {
            gv = P.g[q * W + lane];
            av = P.act[q * W + lane];
            x0 = P.u0[q * W + lane];
            x1 = P.u1[(int64_t)c * W + lane];
            r[j] = gv;
            gv += P.dagg[(int64_t)i * W + lane];
          } else {
            r[j] = 0.f;
          }
        } else {
          if (q < P.cnt) {
            gv = P.g[q * W + lane];
            av = P.act[q * W + lane];
            x0 = P.u0[q * W + lane];
            x1 = P.u1[q * W + lane];
          }
          r[j] = gv;
        }
        dz[jj] = av > 0.f ? gv : 0.f;
        buf[j * BLD + lane] = dz[jj];
        buf[j * BLD + 32 + lane] = x0;
        buf[j * BLD + 64 + lane] = x1;
        db += dz[jj];
      }
      // B of dW: row 32 q + c (piece q of dz_c), K = item; two items per 32-bit word
#pragma unroll
      for (int jj = 0; jj < 16; jj += 2) {
        const int item = warp * 32 + 16 * half + jj;
        const __nv_bfloat162 hi = __floats2bfloat162_rn(dz[jj], dz[jj + 1]);
        const float2 hf = __bfloat1622float2(hi);
        const __nv_bfloat162 lo = __floats2bfloat162_rn(dz[jj] - hf.x, dz[jj + 1] - hf.y);
        const int ob = (item >> 4) * 2048 + ((item >> 3) & 1) * 128 + (item & 7) * 2;
        const int r1 = 32 + lane;
        *reinterpret_cast<__nv_bfloat162*>(Bg + ob + (lane >> 3) * 256 + (lane & 7) * 16) = hi;
        *reinterpret_cast<__nv_bfloat162*>(Bg + ob + (r1 >> 3) * 256 + (r1 & 7) * 16) = lo;
      }
    }
    fence_proxy_async();  // B of dW written through the generic proxy
    __syncwarp();
    {  // A of du: this thread's item, dz in three pieces (K = 32: 16 columns each)
      float x[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) x[k] = buf[lane * BLD + k];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        uint32_t wd[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
          const float2 f = __bfloat1622float2(b);
          x[2 * j] -= f.x;
          x[2 * j + 1] -= f.y;
          wd[j] = *reinterpret_cast<const uint32_t*>(&b);
        }
        tmem_st16(tl + B_ADU + (uint32_t)(16 * p), wd);
      }
    }
    __syncthreads();  // every warp's rows are in the buffers
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {  // A of dW: input gk of the tile's items, piece gp
      uint32_t wd[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int item = 64 * h2 + 2 * c;
        const float* rowp = bufs + (item >> 5) * 32 * BLD + (item & 31) * BLD + 32 + gk;
        const float v0 = rowp[0], v1 = rowp[BLD];
        __nv_bfloat162 b = __floats2bfloat162_rn(v0, v1);
        if (gp) {
          const float2 f = __bfloat1622float2(b);
          b = __floats2bfloat162_rn(v0 - f.x, v1 - f.y);
        }
        wd[c] = *reinterpret_cast<const uint32_t*>(&b);
      }
      tmem_st32(tl + B_AG + (uint32_t)(32 * h2), wd);
    }
    tmem_st_wait();
    tc_before();
    __syncthreads();
    if (tid == 0) {
      tc_after();
      const uint32_t id = idesc_bf16(TT, 64);
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
          mma_bf16(tb + B_DDU, tb + B_ADU + (uint32_t)(16 * p + 8 * ks),
                   desc_nosw(smem_u32(Bdu + ks * 2048), 128, 256), id, (p | ks) != 0 ? 1u : 0u);
#pragma unroll
      for (int ks = 0; ks < 8; ++ks)
        mma_bf16(tb + B_DG, tb + B_AG + (uint32_t)(8 * ks), desc_nosw(smem_u32(Bg + ks * 2048), 128, 256),
                 id, (it > 0 || ks > 0) ? 1u : 0u);
      mma_commit_to(&s_mma);
    }
    const bool done = mbar_wait_bounded(&s_mma, (uint32_t)(it & 1));
    if (__syncthreads_or(!done)) {
      if (tid == 0) set_error(P.status, RBO_ERR_TIMEOUT, 43);
      ok = false;
      break;
    }
    tc_after();
    {  // du rows into buffer columns 32..95 (u is no longer read)
      uint32_t z[32];
      tmem_ld32(tl + B_DDU, z);
#pragma unroll
      for (int c = 0; c < 32; ++c) buf[lane * BLD + 32 + c] = __uint_as_float(z[c]);
      tmem_ld32(tl + B_DDU + 32, z);
#pragma unroll
      for (int c = 0; c < 32; ++c) buf[lane * BLD + 64 + c] = __uint_as_float(z[c]);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (q0 + j < P.cnt) {
        P.out0[(q0 + j) * W + lane] = r[j] + buf[j * BLD + 32 + lane];
        P.out1[(q0 + j) * W + lane] = buf[j * BLD + 64 + lane];
      }
    }
  }
  if (MSG && __any_sync(0xffffffffu, bad) && lane == 0) set_error(P.status, RBO_ERR_ARG, 44);
  if (ok) {
    // this thread's dW^T row summed over the pieces of dz; the hi and lo pieces of u sit
    // in warps (0, 1) and (2, 3)
    uint32_t z0[32], z1[32];
    tmem_ld32(tl + B_DG, z0);
    tmem_ld32(tl + B_DG + 32, z1);
    float sg[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) sg[c] = __uint_as_float(z0[c]) + __uint_as_float(z1[c]);
    __syncthreads();  // every buffer read of the last tile is done
    float* sc = bufs;  // 64 x 33 floats
    if (gp == 1) {
#pragma unroll
      for (int c = 0; c < 32; ++c) sc[gk * 33 + c] = sg[c];
    }
    s_db[warp][lane] = db;
    __syncthreads();
    float* part = P.part + (int64_t)blockIdx.x * (65 * 32);
    if (gp == 0) {
#pragma unroll
      for (int c = 0; c < 32; ++c) part[gk * 32 + c] = sg[c] + sc[gk * 33 + c];
    }
    if (warp == 0) part[64 * 32 + lane] = s_db[0][lane] + s_db[1][lane] + s_db[2][lane] + s_db[3][lane];
  }
  // every product issued has completed before the tensor memory is freed
  if (tid == 0) {
    mma_commit_to(&s_fin);
    mbar_wait_bounded(&s_fin, 0u);
  }
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(BCOLS));
  }
}

static int tc_grid(int64_t items) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (items + TT - 1) / TT;
  return (int)std::min<int64_t>(tiles, (int64_t)TCTAS * std::max(sms, 1));
}

int message_tc_launch(int64_t nnz, int64_t n, const int32_t* col, const float* ein, const float* x,
                      float* e0out, const float* h, const __nv_bfloat16* w, int l, float* m,
                      float* eout, float* pe, DevStatus* status, cudaStream_t st) {
  if (nnz <= 0) return RBO_OK;
  const MsgArgs P{nnz, n, col, ein, x, e0out, h, w, l, m, eout, pe, status};
  const int G = tc_grid(nnz);
  if (!ein && pe)
    message_tc_kernel<true, true><<<G, TNT, TSMEM, st>>>(P);
  else if (!ein)
    message_tc_kernel<true, false><<<G, TNT, TSMEM, st>>>(P);
  else if (pe)
    message_tc_kernel<false, true><<<G, TNT, TSMEM, st>>>(P);
  else
    message_tc_kernel<false, false><<<G, TNT, TSMEM, st>>>(P);
  return note_cuda(cudaGetLastError());
}

int node_update_tc_launch(int64_t n, const int32_t* rowptr, const float* m, const float* hin,
                          const __nv_bfloat16* w, int l, float* agg, float* rh, float* hout,
                          float* sdec, float* tdec, DevStatus* status, cudaStream_t st) {
  if (n <= 0) return RBO_OK;
  node_update_tc_kernel<<<tc_grid(n), TNT, TSMEM, st>>>(n, rowptr, m, hin, w, l, agg, rh, hout, sdec,
                                                        tdec, status);
  return note_cuda(cudaGetLastError());
}

// Backward of layer l (message or node update); *nblocks = CTAs = partials written
int layer_back_tc_launch(bool msg, int64_t cnt, int64_t n, const int32_t* erow, const int32_t* col,
                         const float* g, const float* dagg, const float* act, const float* u0,
                         const float* u1, const __nv_bfloat16* w, int off_w, float* out0, float* out1,
                         float* part, int max_blocks, DevStatus* status, cudaStream_t st,
                         int* nblocks) {
  *nblocks = 0;
  if (cnt <= 0) return RBO_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (cnt + TT - 1) / TT;
  const int G = (int)std::min<int64_t>(std::min<int64_t>(tiles, 2 * (int64_t)std::max(sms, 1)),
                                        (int64_t)max_blocks);
  BackArgs P{cnt, n, erow, col, g, dagg, act, u0, u1, w, off_w, out0, out1, part, status};
  cudaError_t e;
  if (msg) {
    e = cudaFuncSetAttribute(layer_back_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, BSMEM);
    if (e == cudaSuccess) layer_back_tc_kernel<true><<<G, TNT, BSMEM, st>>>(P);
  } else {
    e = cudaFuncSetAttribute(layer_back_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, BSMEM);
    if (e == cudaSuccess) layer_back_tc_kernel<false><<<G, TNT, BSMEM, st>>>(P);
  }
  if (e != cudaSuccess) return note_cuda(e);
  *nblocks = G;
  return note_cuda(cudaGetLastError());
}

}  // namespace gnn
}  // namespace rbo

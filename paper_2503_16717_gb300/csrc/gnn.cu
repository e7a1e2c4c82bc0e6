// Learned sparse-approximate-inverse preconditioner: a 3-layer message-passing
// network (width 32, BF16 weights, FP32 activations and accumulation) that maps the
// entries of A to the values of a right preconditioner M on A's own pattern, with
// hand-written forward, backward and Adam kernels.
//
// Graph: nodes = rows of A; every stored entry (i, j) is an edge carrying a message
// from node j to node i.  Ahat = D^{-1} A.
//   f_i  = [sum_{j!=i} |Ahat_ij|, sum_{j!=i} |Ahat_ji|]
//   x_ij = [Ahat_ij, Ahat_ji, [i == j]]
//   h0 = relu(Wn f + bn), e0 = relu(We x + be)
//   layer: m_ij = relu(Wm [e_ij; h_j] + bm); agg_i = sum_j m_ij;
//          h_i += relu(Wh [h_i; agg_i] + bh); e_ij += m_ij
//   M_ij = (wo . [e_ij; h_i; h_j] + bo + [i == j]) / A_ii
// Loss over residual columns r_k: mean_k ||r_k - A M r_k||^2 / ||r_k||^2.
//
// The message and node-update layers and their backward run on the tensor cores
// (gnn_tc.cu).  The other kernels here give one warp to one node or edge with lane =
// channel (width 32 = warp size); their matrix-vector products broadcast the input
// channels with shuffles.  Every sum
// over edges or nodes runs in a fixed order (rows in CSR order, per-block partials
// reduced in block order), so results are reproducible.  The pattern of A must be
// structurally symmetric (the transpose of edge (i, j) is located by binary search
// in row j); stencil matrices are.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "gnn_params.cuh"

namespace rbo {
namespace gnn {

__device__ __forceinline__ float bf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }
__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// ---- graph construction ---------------------------------------------------------------
// per row: row id of every edge, diagonal value, position of (j, i) for every (i, j)
__global__ void graph_edges_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ col, const double* __restrict__ val,
                                   int32_t* __restrict__ erow, int32_t* __restrict__ tpos,
                                   double* __restrict__ dinv, DevStatus* status) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int beg = rowptr[i], end = rowptr[i + 1];
  double dia = 0.0;
  for (int e = beg; e < end; ++e) {
    erow[e] = (int32_t)i;
    const int j = col[e];
    if (j == (int)i) dia = val[e];
    // binary search for column i in row j (columns sorted)
    int lo = rowptr[j], hi = rowptr[j + 1] - 1, pos = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int cm = col[mid];
      if (cm == (int)i) { pos = mid; break; }
      if (cm < (int)i) lo = mid + 1; else hi = mid - 1;
    }
    tpos[e] = pos;
    if (pos < 0) set_error(status, RBO_ERR_ARG, 20);
  }
  if (dia == 0.0) set_error(status, RBO_ERR_ARG, 21);
  dinv[i] = dia != 0.0 ? 1.0 / dia : 0.0;
}

__global__ void graph_features_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                      const int32_t* __restrict__ col, const double* __restrict__ val,
                                      const int32_t* __restrict__ tpos, const double* __restrict__ dinv,
                                      float* __restrict__ x, float* __restrict__ f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double rs = 0.0, cs = 0.0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int j = col[e];
    const double ah = val[e] * dinv[i];
    const double aht = tpos[e] >= 0 ? val[tpos[e]] * dinv[j] : 0.0;
    x[3 * (int64_t)e + 0] = (float)ah;
    x[3 * (int64_t)e + 1] = (float)aht;
    x[3 * (int64_t)e + 2] = (j == (int)i) ? 1.f : 0.f;
    if (j != (int)i) {
      rs += fabs(ah);
      cs += fabs(aht);
    }
  }
  f[2 * i] = (float)rs;
  f[2 * i + 1] = (float)cs;
}

// ---- forward ------------------------------------------------------------------------
// h[i][c] = relu(Wn[c] . f_i + bn[c])  and  e[e][c] = relu(We[c] . x_e + be[c])
__global__ void encode_kernel(int64_t cnt, int nin, const float* __restrict__ in,
                              const __nv_bfloat16* __restrict__ w, int off_w, int off_b,
                              float* __restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cnt * W) return;
  const int64_t it = t / W;
  const int c = (int)(t % W);
  float z = bf(w, off_b + c);
  for (int k = 0; k < nin; ++k) z = fmaf(bf(w, off_w + c * nin + k), in[it * nin + k], z);
  out[t] = relu(z);
}

// decoder: M_e = (wo . [e; h_i; h_j] + bo + [i == j]) / A_ii from the terms the last
// layers left: pe_e = wo[0:32] . e (message layer), s_i = wo[32:64] . h_i and
// t_j = wo[64:96] . h_j (node update); thread per edge
__global__ void decode_terms_kernel(int64_t nnz, const int32_t* __restrict__ erow,
                                    const int32_t* __restrict__ col, const float* __restrict__ pe,
                                    const float* __restrict__ sdec, const float* __restrict__ tdec,
                                    const __nv_bfloat16* __restrict__ w, const double* __restrict__ dinv,
                                    double* __restrict__ Mval) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nnz) return;
  const int i = erow[q], j = col[q];
  const float out = pe[q] + sdec[i] + tdec[j] + bf(w, OFF_BO) + (i == j ? 1.f : 0.f);
  Mval[q] = (double)out * dinv[i];
}

// ---- loss (float64) ---------------------------------------------------------------------
// Z = Mat R  for a matrix with A's pattern and values `v` (R: n x nr, ld ldr)
__global__ void spmm_kernel(int64_t n, int nr, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, const double* __restrict__ v,
                            const double* __restrict__ R, int64_t ldr, double* __restrict__ Z,
                            int64_t ldz) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nr) return;
  const int64_t i = t % n;
  const int k = (int)(t / n);
  double s = 0.0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s = fma(v[e], R[col[e] + k * ldr], s);
  Z[i + k * ldz] = s;
}

// (A^T Y)_i = sum over stored (j, i) of A_ji Y_j = sum over row i of A[tpos] Y[col]
__global__ void spmm_t_kernel(int64_t n, int nr, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, const int32_t* __restrict__ tpos,
                              const double* __restrict__ v, const double* __restrict__ Y,
                              int64_t ldy, double* __restrict__ Z, int64_t ldz) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nr) return;
  const int64_t i = t % n;
  const int k = (int)(t / n);
  double s = 0.0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s = fma(v[tpos[e]], Y[col[e] + k * ldy], s);
  Z[i + k * ldz] = s;
}

// per-block partial sums of ||R_k - Y_k||^2 and ||R_k||^2 ; E = R - Y written to Y
__global__ void residual_norms_kernel(int64_t n, int nr, const double* __restrict__ R, int64_t ldr,
                                      double* __restrict__ Y, int64_t ldy, double* __restrict__ part) {
  __shared__ double red[2][256];
  const int k = blockIdx.y;
  double se = 0.0, sr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r = R[i + k * ldr];
    const double e = r - Y[i + k * ldy];
    Y[i + k * ldy] = e;
    se = fma(e, e, se);
    sr = fma(r, r, sr);
  }
  red[0][threadIdx.x] = se;
  red[1][threadIdx.x] = sr;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * ((int64_t)k * gridDim.x + blockIdx.x)] = red[0][0];
    part[2 * ((int64_t)k * gridDim.x + blockIdx.x) + 1] = red[1][0];
  }
}

__global__ void scale_cols_kernel(int64_t n, int nr, double* __restrict__ Y, int64_t ldy,
                                  const double* __restrict__ colscale) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * nr) return;
  const int64_t i = t % n;
  const int k = (int)(t / n);
  Y[i + k * ldy] *= colscale[k];
}

// dM_e = sum_k dZ[row_e][k] R[col_e][k]; dout_e = dM_e / A_ii (float)
__global__ void dm_kernel(int64_t nnz, int nr, const int32_t* __restrict__ erow,
                          const int32_t* __restrict__ col, const double* __restrict__ dZ,
                          int64_t ldz, const double* __restrict__ R, int64_t ldr,
                          const double* __restrict__ dinv, float* __restrict__ dout) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nnz) return;
  const int i = erow[q], j = col[q];
  double s = 0.0;
  for (int k = 0; k < nr; ++k) s = fma(dZ[i + k * ldz], R[j + k * ldr], s);
  dout[q] = (float)(s * dinv[i]);
}

// ---- backward ----------------------------------------------------------------------------
// Weight-gradient partials: every block writes its partial sum of one weight group to
// part[blockIdx][0..cnt) (fixed order), reduced by reduce_partials_kernel.
__device__ __forceinline__ void block_partial_store(float* acc, int cnt, float* smem_red,
                                                    float* part) {
  // acc: per-warp values, lane-major: acc[k] belongs to (lane, k); reduce over warps
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per_lane = cnt / 32;
  for (int k = 0; k < per_lane; ++k) smem_red[(warp * per_lane + k) * 32 + lane] = acc[k];
  __syncthreads();
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int k = t / 32, ln = t % 32;
    float s = 0.f;
    for (int w2 = 0; w2 < nw; ++w2) s += smem_red[(w2 * per_lane + k) * 32 + ln];
    part[(int64_t)blockIdx.x * cnt + t] = s;
  }
  __syncthreads();
}

// decoder backward: grad wo/bo partials, de (edges), dh (nodes)
__global__ void decode_back_edges_kernel(int64_t nnz, const int32_t* __restrict__ erow,
                                         const int32_t* __restrict__ col, const float* __restrict__ e,
                                         const float* __restrict__ h, const float* __restrict__ dout,
                                         const __nv_bfloat16* __restrict__ w, float* __restrict__ de,
                                         float* __restrict__ part) {
  extern __shared__ float sred[];
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float w0 = bf(w, OFF_WO + lane);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};  // g_wo[lane], g_wo[32+lane], g_wo[64+lane], g_bo (lane 0)
  // edges warp0, warp0 + nwarps, ... in order, the loads of 4 of them issued together
  for (int64_t q0 = warp0; q0 < nnz; q0 += 4 * nwarps) {
    float d[4], ev[4], hi[4], hj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t q = q0 + u * nwarps;
      const bool v = q < nnz;
      const int i = v ? erow[q] : 0, j = v ? col[q] : 0;
      d[u] = v ? dout[q] : 0.f;
      ev[u] = v ? e[q * W + lane] : 0.f;
      hi[u] = v ? h[(int64_t)i * W + lane] : 0.f;
      hj[u] = v ? h[(int64_t)j * W + lane] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t q = q0 + u * nwarps;
      if (q < nnz) {
        acc[0] = fmaf(d[u], ev[u], acc[0]);
        acc[1] = fmaf(d[u], hi[u], acc[1]);
        acc[2] = fmaf(d[u], hj[u], acc[2]);
        if (lane == 0) acc[3] += d[u];
        de[q * W + lane] = d[u] * w0;
      }
    }
  }
  block_partial_store(acc, 128, sred, part);
}

// dh_i = wo[32:64] * sum_{e in row i} dout_e + wo[64:96] * sum_{e in row i} dout_{tpos e}
__global__ void decode_back_nodes_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                         const int32_t* __restrict__ tpos,
                                         const float* __restrict__ dout,
                                         const __nv_bfloat16* __restrict__ w, float* __restrict__ dh) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * W) return;
  const int64_t i = t / W;
  const int c = (int)(t % W);
  float s1 = 0.f, s2 = 0.f;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    s1 += dout[e];
    s2 += dout[tpos[e]];
  }
  dh[t] = bf(w, OFF_WO + W + c) * s1 + bf(w, OFF_WO + 2 * W + c) * s2;
}

// dh_l[i] += sum over row i of dhj[tpos e]  (the column scatter, gathered per node)
__global__ void gather_cols_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ tpos, const float* __restrict__ dhj,
                                   float* __restrict__ dhl) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * W) return;
  const int64_t i = t / W;
  const int c = (int)(t % W);
  float s = dhl[t];
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s += dhj[(int64_t)tpos[e] * W + c];
  dhl[t] = s;
}

// encoder backward: dz = d * [out > 0]; g_W[c][k] += dz x_k, g_b[c] += dz (NIN inputs per
// item); lane = channel c, warp w handles items w, w + nw, ... in order, the loads of 4
// items issued together; blocks stride over items
template <int NIN>
__device__ __forceinline__ void encode_back_body(int64_t cnt, const float* __restrict__ in,
                                                 const float* __restrict__ out,
                                                 const float* __restrict__ d, float* __restrict__ part,
                                                 float* sred) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float acc[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k] = 0.f;
  for (int64_t it0 = warp0; it0 < cnt; it0 += 4 * nwarps) {
    float dz[4], x[4][NIN];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t it = it0 + u * nwarps;
      const bool v = it < cnt;
      const float o = v ? out[it * W + lane] : 0.f;
      const float g = v ? d[it * W + lane] : 0.f;
      dz[u] = o > 0.f ? g : 0.f;
#pragma unroll
      for (int k = 0; k < NIN; ++k) x[u][k] = v ? in[it * NIN + k] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < NIN; ++k) acc[k] = fmaf(dz[u], x[u][k], acc[k]);
      acc[NIN] += dz[u];
    }
  }
  block_partial_store(acc, 32 * 32, sred, part);
}
// edge encoder (3 features per edge) and node encoder (2 features per node)
__global__ void encode_back_edges_kernel(int64_t cnt, const float* __restrict__ in,
                                         const float* __restrict__ out, const float* __restrict__ d,
                                         float* __restrict__ part) {
  extern __shared__ float sred[];
  encode_back_body<3>(cnt, in, out, d, part, sred);
}
__global__ void encode_back_nodes_kernel(int64_t cnt, const float* __restrict__ in,
                                         const float* __restrict__ out, const float* __restrict__ d,
                                         float* __restrict__ part) {
  extern __shared__ float sred[];
  encode_back_body<2>(cnt, in, out, d, part, sred);
}

// grad[dst[k]] = sum over blocks of part[b][src[k]]: one warp per output, lane l adds
// blocks l, l + 32, ... in order, then a fixed butterfly over the lanes (deterministic)
__global__ void reduce_partials_kernel(const float* __restrict__ part, int nblocks, int cnt,
                                       const int* __restrict__ map_src, const int* __restrict__ map_dst,
                                       int nmap, float* __restrict__ grad) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (t >= nmap) return;
  const int s = map_src[t];
  float acc = 0.f;
  for (int b = lane; b < nblocks; b += 32) acc += part[(int64_t)b * cnt + s];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) grad[map_dst[t]] = acc;
}

__global__ void adam_kernel(int np, float* __restrict__ th, const float* __restrict__ g,
                            float* __restrict__ m1, float* __restrict__ m2, float lr, float b1,
                            float b2, float eps, float c1, float c2, __nv_bfloat16* __restrict__ wbf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  const float gg = g[t];
  const float a = b1 * m1[t] + (1.f - b1) * gg;
  const float v = b2 * m2[t] + (1.f - b2) * gg * gg;
  m1[t] = a;
  m2[t] = v;
  const float x = th[t] - lr * (a / c1) / (sqrtf(v / c2) + eps);
  th[t] = x;
  wbf[t] = __float2bfloat16_rn(x);
}

__global__ void to_bf16_kernel(int np, const float* __restrict__ th, __nv_bfloat16* __restrict__ wbf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < np) wbf[t] = __float2bfloat16_rn(th[t]);
}

}  // namespace gnn
}  // namespace rbo

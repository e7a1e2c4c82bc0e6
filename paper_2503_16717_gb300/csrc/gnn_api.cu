// Host side of the learned-SPAI network: model handle, forward (inference), loss and
// gradient, Adam training step, and s-step GMRES with the resulting right
// preconditioner.  Kernels are in gnn.cu.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "gnn_params.cuh"
#include "rbo_internal.cuh"

namespace rbo {
namespace gnn {

// kernels (gnn.cu)
__global__ void graph_edges_kernel(int64_t, const int32_t*, const int32_t*, const double*, int32_t*,
                                   int32_t*, double*, DevStatus*);
__global__ void graph_features_kernel(int64_t, const int32_t*, const int32_t*, const double*,
                                      const int32_t*, const double*, float*, float*);
__global__ void encode_kernel(int64_t, int, const float*, const __nv_bfloat16*, int, int, float*);
// tensor-core message and node-update layers (gnn_tc.cu)
int message_tc_launch(int64_t nnz, int64_t n, const int32_t* col, const float* ein, const float* x,
                      float* e0out, const float* h, const __nv_bfloat16* w, int l, float* m,
                      float* eout, float* pe, DevStatus* status, cudaStream_t st);
int node_update_tc_launch(int64_t n, const int32_t* rowptr, const float* m, const float* hin,
                          const __nv_bfloat16* w, int l, float* agg, float* rh, float* hout,
                          float* sdec, float* tdec, DevStatus* status, cudaStream_t st);
__global__ void decode_terms_kernel(int64_t, const int32_t*, const int32_t*, const float*, const float*,
                                    const float*, const __nv_bfloat16*, const double*, double*);
__global__ void spmm_kernel(int64_t, int, const int32_t*, const int32_t*, const double*,
                            const double*, int64_t, double*, int64_t);
__global__ void spmm_t_kernel(int64_t, int, const int32_t*, const int32_t*, const int32_t*,
                              const double*, const double*, int64_t, double*, int64_t);
__global__ void residual_norms_kernel(int64_t, int, const double*, int64_t, double*, int64_t,
                                      double*);
__global__ void scale_cols_kernel(int64_t, int, double*, int64_t, const double*);
__global__ void dm_kernel(int64_t, int, const int32_t*, const int32_t*, const double*, int64_t,
                          const double*, int64_t, const double*, float*);
__global__ void decode_back_edges_kernel(int64_t, const int32_t*, const int32_t*, const float*,
                                         const float*, const float*, const __nv_bfloat16*, float*,
                                         float*);
__global__ void decode_back_nodes_kernel(int64_t, const int32_t*, const int32_t*, const float*,
                                         const __nv_bfloat16*, float*);
int layer_back_tc_launch(bool msg, int64_t cnt, int64_t n, const int32_t* erow, const int32_t* col,
                         const float* g, const float* dagg, const float* act, const float* u0,
                         const float* u1, const __nv_bfloat16* w, int off_w, float* out0, float* out1,
                         float* part, int max_blocks, DevStatus* status, cudaStream_t st,
                         int* nblocks);
__global__ void gather_cols_kernel(int64_t, const int32_t*, const int32_t*, const float*, float*);
__global__ void encode_back_edges_kernel(int64_t, const float*, const float*, const float*, float*);
__global__ void encode_back_nodes_kernel(int64_t, const float*, const float*, const float*, float*);
__global__ void reduce_partials_kernel(const float*, int, int, const int*, const int*, int, float*);
__global__ void adam_kernel(int, float*, const float*, float*, float*, float, float, float, float,
                            float, float, __nv_bfloat16*);
__global__ void to_bf16_kernel(int, const float*, __nv_bfloat16*);

// gradient-reduction maps: (index inside a block partial) -> (parameter index)
struct Map {
  int* src = nullptr;
  int* dst = nullptr;
  int cnt = 0;      // partial length per block
  int nmap = 0;
};

}  // namespace gnn
}  // namespace rbo

struct rbo_gnn_s {
  int device = -1;
  float* theta = nullptr;
  __nv_bfloat16* wbf = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grad = nullptr;
  int step = 0;
  rbo::gnn::Map dec, layer_node[rbo::gnn::NL], layer_msg[rbo::gnn::NL], enc_e, enc_n;
  int* maps_dev = nullptr;
};

namespace rbo {
namespace gnn {

constexpr int BLK = 128;       // threads of the backward reduction kernels (4 warps)
constexpr int NBLK_RED = 600;  // blocks of the backward reduction kernels

static uint64_t sm64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// He-like initial weights from the SplitMix64 stream (Box-Muller normals); output
// layer and biases zero, so an untrained network is the Jacobi preconditioner.
static void init_host(uint64_t seed, std::vector<float>& th) {
  th.assign(NPARAM, 0.f);
  uint64_t s = seed;
  auto normal = [&]() {
    double u1 = ((sm64(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    double u2 = (sm64(s) >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  auto fill = [&](int off, int rows, int cols) {
    const double sc = 0.5 * std::sqrt(2.0 / cols);
    for (int t = 0; t < rows * cols; ++t) th[off + t] = (float)(normal() * sc);
  };
  fill(OFF_WN, W, 2);
  fill(OFF_WE, W, 3);
  for (int l = 0; l < NL; ++l) {
    fill(off_wm(l), W, 2 * W);
    fill(off_wh(l), W, 2 * W);
  }
}

static int build_maps(rbo_gnn_s* g) {
  std::vector<int> all;
  struct Spec { Map* m; std::vector<int> src, dst; int cnt; };
  std::vector<Spec> specs;
  {  // decoder: (lane, k) at k*32+lane: k=0..2 -> wo[k*32+lane], (0,3) -> bo
    Spec s{&g->dec, {}, {}, 128};
    for (int k = 0; k < 3; ++k)
      for (int ln = 0; ln < W; ++ln) { s.src.push_back(k * 32 + ln); s.dst.push_back(OFF_WO + k * W + ln); }
    s.src.push_back(3 * 32 + 0);
    s.dst.push_back(OFF_BO);
    specs.push_back(s);
  }
  for (int l = 0; l < NL; ++l) {
    for (int which = 0; which < 2; ++which) {
      Spec s{which == 0 ? &g->layer_node[l] : &g->layer_msg[l], {}, {}, 65 * 32};
      const int ow = which == 0 ? off_wh(l) : off_wm(l);
      const int ob = which == 0 ? off_bh(l) : off_bm(l);
      for (int ln = 0; ln < W; ++ln) {
        for (int k = 0; k < 2 * W; ++k) { s.src.push_back(k * 32 + ln); s.dst.push_back(ow + ln * 2 * W + k); }
        s.src.push_back(2 * W * 32 + ln);
        s.dst.push_back(ob + ln);
      }
      specs.push_back(s);
    }
  }
  for (int which = 0; which < 2; ++which) {  // edge encoder (3 inputs), node encoder (2)
    const int nin = which == 0 ? 3 : 2;
    Spec s{which == 0 ? &g->enc_e : &g->enc_n, {}, {}, 32 * 32};
    const int ow = which == 0 ? OFF_WE : OFF_WN, ob = which == 0 ? OFF_BE : OFF_BN;
    for (int ln = 0; ln < W; ++ln) {
      for (int k = 0; k < nin; ++k) { s.src.push_back(k * 32 + ln); s.dst.push_back(ow + ln * nin + k); }
      s.src.push_back(nin * 32 + ln);
      s.dst.push_back(ob + ln);
    }
    specs.push_back(s);
  }
  size_t tot = 0;
  for (auto& s : specs) tot += 2 * s.src.size();
  if (cudaMalloc(&g->maps_dev, tot * sizeof(int)) != cudaSuccess) return RBO_ERR_NOMEM;
  std::vector<int> host;
  host.reserve(tot);
  for (auto& s : specs) {
    s.m->cnt = s.cnt;
    s.m->nmap = (int)s.src.size();
    s.m->src = g->maps_dev + host.size();
    host.insert(host.end(), s.src.begin(), s.src.end());
    s.m->dst = g->maps_dev + host.size();
    host.insert(host.end(), s.dst.begin(), s.dst.end());
  }
  return note_cuda(cudaMemcpy(g->maps_dev, host.data(), tot * sizeof(int), cudaMemcpyHostToDevice));
}

// device buffers of one call
struct Work {
  int64_t n = 0, nnz = 0;
  int nr = 0;
  int32_t *erow = nullptr, *tpos = nullptr;
  double* dinv = nullptr;
  float *x = nullptr, *f = nullptr;
  float *e[NL + 1] = {}, *h[NL + 1] = {}, *m[NL] = {}, *agg[NL] = {}, *rh[NL] = {};
  double* Mval = nullptr;
  float *pe = nullptr, *sdec = nullptr, *tdec = nullptr;  // decoder terms of the last layer
  // loss / backward
  double *Z = nullptr, *Y = nullptr, *dZ = nullptr, *npart = nullptr, *cscale = nullptr;
  float *dout = nullptr, *de = nullptr, *de2 = nullptr, *dhj = nullptr, *dh = nullptr, *dh2 = nullptr,
        *dagg = nullptr, *part = nullptr;
};

static size_t work_bytes(int64_t n, int64_t nnz, int nr, bool train) {
  size_t b = 0;
  b += (size_t)nnz * 8 + (size_t)n * 8 + (size_t)nnz * 12 + (size_t)n * 8;
  const int ne = train ? NL + 1 : 2, nm = train ? NL : 1;
  b += (size_t)ne * nnz * W * 4 + (size_t)ne * n * W * 4;
  b += (size_t)nm * nnz * W * 4 + (size_t)2 * nm * n * W * 4;
  b += (size_t)nnz * 8;
  b += (size_t)nnz * 4 + (size_t)2 * n * 4;
  if (train) {
    b += 3 * (size_t)n * nr * 8 + 2 * (size_t)nr * 1024 * 8 + 64 * 8;
    b += (size_t)nnz * 4 + 3 * (size_t)nnz * W * 4 + 3 * (size_t)n * W * 4;
    b += (size_t)NBLK_RED * 65 * 32 * 4;
  }
  return b + 64 * 4096;
}

static int work_take(Arena* ar, Work& w, int64_t n, int64_t nnz, int nr, bool train) {
  w.n = n;
  w.nnz = nnz;
  w.nr = nr;
  auto T = [&](size_t bytes) { return ar->take(std::max<size_t>(bytes, 16)); };
  w.erow = (int32_t*)T(nnz * 4);
  w.tpos = (int32_t*)T(nnz * 4);
  w.dinv = (double*)T(n * 8);
  w.x = (float*)T(nnz * 12);
  w.f = (float*)T(n * 8);
  const int ne = train ? NL + 1 : 2, nm = train ? NL : 1;
  for (int l = 0; l < ne; ++l) {
    w.e[l] = (float*)T(nnz * W * 4);
    w.h[l] = (float*)T(n * W * 4);
  }
  for (int l = 0; l < nm; ++l) {
    w.m[l] = (float*)T(nnz * W * 4);
    w.agg[l] = (float*)T(n * W * 4);
    w.rh[l] = (float*)T(n * W * 4);
  }
  w.Mval = (double*)T(nnz * 8);
  w.pe = (float*)T(nnz * 4);
  w.sdec = (float*)T(n * 4);
  w.tdec = (float*)T(n * 4);
  if (train) {
    w.Z = (double*)T((size_t)n * nr * 8);
    w.Y = (double*)T((size_t)n * nr * 8);
    w.dZ = (double*)T((size_t)n * nr * 8);
    w.npart = (double*)T((size_t)2 * nr * 1024 * 8);
    w.cscale = (double*)T(64 * 8);
    w.dout = (float*)T(nnz * 4);
    w.de = (float*)T(nnz * W * 4);
    w.de2 = (float*)T(nnz * W * 4);
    w.dhj = (float*)T(nnz * W * 4);
    w.dh = (float*)T(n * W * 4);
    w.dh2 = (float*)T(n * W * 4);
    w.dagg = (float*)T(n * W * 4);
    w.part = (float*)T((size_t)NBLK_RED * 65 * 32 * 4);
    if (!w.Z || !w.Y || !w.dZ || !w.npart || !w.cscale || !w.dout || !w.de || !w.de2 || !w.dhj ||
        !w.dh || !w.dh2 || !w.dagg || !w.part)
      return RBO_ERR_NOMEM;
  }
  if (!w.erow || !w.tpos || !w.dinv || !w.x || !w.f || !w.Mval || !w.pe || !w.sdec || !w.tdec)
    return RBO_ERR_NOMEM;
  for (int l = 0; l < ne; ++l)
    if (!w.e[l] || !w.h[l]) return RBO_ERR_NOMEM;
  for (int l = 0; l < nm; ++l)
    if (!w.m[l] || !w.agg[l] || !w.rh[l]) return RBO_ERR_NOMEM;
  return RBO_OK;
}

static unsigned grid1(int64_t threads, int bs = 256) {
  int64_t b = (threads + bs - 1) / bs;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 30));
}

// graph + forward; with train == false only two activation buffers are kept, and only
// what the next layer reads is written.  The edge encoder runs inside the first message
// layer; the decoder's dot products inside the last message and node layers.
static int forward(rbo_gnn_s* g, const rbo_csr* A, Work& w, Arena* ar, cudaStream_t st, bool train,
                   int* launches) {
  const int64_t n = A->n, nnz = A->nnz;
  graph_edges_kernel<<<grid1(n), 256, 0, st>>>(n, A->rowptr, A->col, A->val, w.erow, w.tpos, w.dinv,
                                               ar->status);
  graph_features_kernel<<<grid1(n), 256, 0, st>>>(n, A->rowptr, A->col, A->val, w.tpos, w.dinv, w.x,
                                                  w.f);
  encode_kernel<<<grid1(n * W), 256, 0, st>>>(n, 2, w.f, g->wbf, OFF_WN, OFF_BN, w.h[0]);
  *launches += 3;
  for (int l = 0; l < NL; ++l) {
    const int a = train ? l : (l & 1), b = train ? l + 1 : ((l + 1) & 1);
    const bool last = l == NL - 1;
    float* mm = train ? w.m[l] : w.m[0];
    float* ag = train ? w.agg[l] : nullptr;
    float* rr = train ? w.rh[l] : nullptr;
    float* eo = (train || !last) ? w.e[b] : nullptr;
    float* ho = (train || !last) ? w.h[b] : nullptr;
    int rc = message_tc_launch(nnz, n, A->col, l == 0 ? nullptr : w.e[a], w.x,
                               (l == 0 && train) ? w.e[0] : nullptr, w.h[a], g->wbf, l, mm, eo,
                               last ? w.pe : nullptr, ar->status, st);
    if (rc == RBO_OK)
      rc = node_update_tc_launch(n, A->rowptr, mm, w.h[a], g->wbf, l, ag, rr, ho,
                                 last ? w.sdec : nullptr, last ? w.tdec : nullptr, ar->status, st);
    if (rc != RBO_OK) return rc;
    *launches += 2;
  }
  decode_terms_kernel<<<grid1(nnz), 256, 0, st>>>(nnz, w.erow, A->col, w.pe, w.sdec, w.tdec, g->wbf,
                                                  w.dinv, w.Mval);
  *launches += 1;
  return note_cuda(cudaGetLastError());
}

static void reduce_group(const Map& m, const float* part, float* grad, cudaStream_t st,
                         int nblocks = NBLK_RED) {
  reduce_partials_kernel<<<grid1((int64_t)m.nmap * 32), 256, 0, st>>>(part, nblocks, m.cnt, m.src, m.dst, m.nmap,
                                                        grad);
}

// loss and gradient into g->grad; returns the loss on the host
static int loss_grad(rbo_gnn_s* g, const rbo_csr* A, const double* R, int nr, int64_t ldr,
                     double* loss, Arena** arp, cudaStream_t st, int* launches) {
  const int64_t n = A->n, nnz = A->nnz;
  Arena* ar = nullptr;
  int e = arena_prepare(&ar, work_bytes(n, nnz, nr, true));
  if (e) return e;
  if ((e = note_cuda(cudaMemsetAsync(ar->base, 0, 1024, st)))) return e;
  Work w;
  if ((e = work_take(ar, w, n, nnz, nr, true))) return e;
  if ((e = forward(g, A, w, ar, st, true, launches))) return e;
  // Z = M R ; Y = A Z ; E = R - Y (in Y) with per-block norms
  spmm_kernel<<<grid1(n * nr), 256, 0, st>>>(n, nr, A->rowptr, A->col, w.Mval, R, ldr, w.Z, n);
  spmm_kernel<<<grid1(n * nr), 256, 0, st>>>(n, nr, A->rowptr, A->col, A->val, w.Z, n, w.Y, n);
  const int nb = 256;
  residual_norms_kernel<<<dim3(nb, nr), 256, 0, st>>>(n, nr, R, ldr, w.Y, n, w.npart);
  *launches += 3;
  std::vector<double> hp((size_t)2 * nr * nb);
  if ((e = note_cuda(cudaMemcpyAsync(hp.data(), w.npart, hp.size() * 8, cudaMemcpyDeviceToHost, st))))
    return e;
  if ((e = finish_status(ar, st, nullptr))) return e;
  double L = 0.0;
  std::vector<double> cs(nr);
  for (int k = 0; k < nr; ++k) {
    double se = 0.0, sr = 0.0;
    for (int b = 0; b < nb; ++b) {
      se += hp[2 * ((size_t)k * nb + b)];
      sr += hp[2 * ((size_t)k * nb + b) + 1];
    }
    if (!(sr > 0.0)) return RBO_ERR_ARG;
    L += se / sr;
    cs[k] = -2.0 / (sr * nr);
  }
  *loss = L / nr;
  if ((e = note_cuda(cudaMemcpyAsync(w.cscale, cs.data(), nr * 8, cudaMemcpyHostToDevice, st))))
    return e;
  // dY = -2 E w / nr ; dZ = A^T dY ; dM ; dout = dM / A_ii
  scale_cols_kernel<<<grid1(n * nr), 256, 0, st>>>(n, nr, w.Y, n, w.cscale);
  spmm_t_kernel<<<grid1(n * nr), 256, 0, st>>>(n, nr, A->rowptr, A->col, w.tpos, A->val, w.Y, n, w.dZ,
                                               n);
  dm_kernel<<<grid1(nnz), 256, 0, st>>>(nnz, nr, w.erow, A->col, w.dZ, n, R, ldr, w.dinv, w.dout);
  *launches += 3;
  // decoder
  const size_t sm_dec = (size_t)(BLK / 32) * 128 * 4,
               sm_enc = (size_t)(BLK / 32) * 32 * 32 * 4;
  decode_back_edges_kernel<<<NBLK_RED, BLK, sm_dec, st>>>(nnz, w.erow, A->col, w.e[NL], w.h[NL],
                                                          w.dout, g->wbf, w.de, w.part);
  reduce_group(g->dec, w.part, g->grad, st);
  decode_back_nodes_kernel<<<grid1(n * W), 256, 0, st>>>(n, A->rowptr, w.tpos, w.dout, g->wbf, w.dh);
  *launches += 3;
  float *dh = w.dh, *dhn = w.dh2, *de = w.de, *den = w.de2;
  for (int l = NL - 1; l >= 0; --l) {
    int nb = 0;
    if ((e = layer_back_tc_launch(false, n, n, nullptr, nullptr, dh, nullptr, w.rh[l], w.h[l],
                                  w.agg[l], g->wbf, off_wh(l), dhn, w.dagg, w.part, NBLK_RED,
                                  ar->status, st, &nb)))
      return e;
    reduce_group(g->layer_node[l], w.part, g->grad, st, nb);
    if ((e = layer_back_tc_launch(true, nnz, n, w.erow, A->col, de, w.dagg, w.m[l], w.e[l], w.h[l],
                                  g->wbf, off_wm(l), den, w.dhj, w.part, NBLK_RED, ar->status, st,
                                  &nb)))
      return e;
    reduce_group(g->layer_msg[l], w.part, g->grad, st, nb);
    gather_cols_kernel<<<grid1(n * W), 256, 0, st>>>(n, A->rowptr, w.tpos, w.dhj, dhn);
    *launches += 5;
    std::swap(dh, dhn);
    std::swap(de, den);
  }
  encode_back_edges_kernel<<<NBLK_RED, BLK, sm_enc, st>>>(nnz, w.x, w.e[0], de, w.part);
  reduce_group(g->enc_e, w.part, g->grad, st);
  encode_back_nodes_kernel<<<NBLK_RED, BLK, sm_enc, st>>>(n, w.f, w.h[0], dh, w.part);
  reduce_group(g->enc_n, w.part, g->grad, st);
  *launches += 4;
  *arp = ar;
  return note_cuda(cudaGetLastError());
}

static int check_csr(const rbo_csr* A) {
  if (!A || A->n < 1 || !A->rowptr || !A->col || !A->val || A->nnz < 1 || A->nnz >= (1LL << 31))
    return RBO_ERR_ARG;
  return RBO_OK;
}

}  // namespace gnn
}  // namespace rbo

using namespace rbo;
using namespace rbo::gnn;

extern "C" {

int rbo_gnn_param_count(void) { return NPARAM; }

int rbo_gnn_create(uint64_t seed, rbo_gnn* out) {
  if (!out) return RBO_ERR_ARG;
  rbo_gnn_s* g = new (std::nothrow) rbo_gnn_s;
  if (!g) return RBO_ERR_NOMEM;
  cudaGetDevice(&g->device);
  if (cudaMalloc(&g->theta, NPARAM * 4) != cudaSuccess || cudaMalloc(&g->wbf, NPARAM * 2) != cudaSuccess ||
      cudaMalloc(&g->m1, NPARAM * 4) != cudaSuccess || cudaMalloc(&g->m2, NPARAM * 4) != cudaSuccess ||
      cudaMalloc(&g->grad, NPARAM * 4) != cudaSuccess) {
    cudaGetLastError();
    rbo_gnn_destroy(g);
    return RBO_ERR_NOMEM;
  }
  int e = build_maps(g);
  if (e) {
    rbo_gnn_destroy(g);
    return e;
  }
  std::vector<float> th;
  init_host(seed, th);
  e = rbo_gnn_set_params(g, th.data());
  if (e) {
    rbo_gnn_destroy(g);
    return e;
  }
  *out = g;
  return RBO_OK;
}

int rbo_gnn_destroy(rbo_gnn g) {
  if (!g) return RBO_OK;
  cudaFree(g->theta);
  cudaFree(g->wbf);
  cudaFree(g->m1);
  cudaFree(g->m2);
  cudaFree(g->grad);
  cudaFree(g->maps_dev);
  delete g;
  return RBO_OK;
}

int rbo_gnn_set_params(rbo_gnn g, const float* host) {
  if (!g || !host) return RBO_ERR_ARG;
  int e = note_cuda(cudaMemcpy(g->theta, host, NPARAM * 4, cudaMemcpyHostToDevice));
  if (e) return e;
  cudaMemset(g->m1, 0, NPARAM * 4);
  cudaMemset(g->m2, 0, NPARAM * 4);
  g->step = 0;
  to_bf16_kernel<<<grid1(NPARAM), 256>>>(NPARAM, g->theta, g->wbf);
  return note_cuda(cudaDeviceSynchronize());
}

int rbo_gnn_get_params(rbo_gnn g, float* host) {
  if (!g || !host) return RBO_ERR_ARG;
  return note_cuda(cudaMemcpy(host, g->theta, NPARAM * 4, cudaMemcpyDeviceToHost));
}

int rbo_gnn_infer(rbo_gnn g, const rbo_csr* A, double* Mval, void* stream) {
  if (!g || !Mval) return RBO_ERR_ARG;
  int e = check_csr(A);
  if (e) return e;
  cudaStream_t st = (cudaStream_t)stream;
  Arena* ar = nullptr;
  if ((e = arena_prepare(&ar, work_bytes(A->n, A->nnz, 0, false)))) return e;
  if ((e = note_cuda(cudaMemsetAsync(ar->base, 0, 1024, st)))) return e;
  Work w;
  if ((e = work_take(ar, w, A->n, A->nnz, 0, false))) return e;
  int launches = 0;
  if ((e = forward(g, A, w, ar, st, false, &launches))) return e;
  if ((e = note_cuda(cudaMemcpyAsync(Mval, w.Mval, (size_t)A->nnz * 8, cudaMemcpyDeviceToDevice, st))))
    return e;
  return finish_status(ar, st, nullptr);
}

int rbo_gnn_loss_grad(rbo_gnn g, const rbo_csr* A, const double* R, int32_t nr, int64_t ldr,
                      double* loss, float* grad_host, void* stream) {
  if (!g || !R || nr < 1 || nr > 64 || !loss) return RBO_ERR_ARG;
  int e = check_csr(A);
  if (e) return e;
  if (ldr < A->n) return RBO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Arena* ar = nullptr;
  int launches = 0;
  if ((e = loss_grad(g, A, R, nr, ldr, loss, &ar, st, &launches))) return e;
  if (grad_host &&
      (e = note_cuda(cudaMemcpyAsync(grad_host, g->grad, NPARAM * 4, cudaMemcpyDeviceToHost, st))))
    return e;
  return finish_status(ar, st, nullptr);
}

int rbo_gnn_train_step(rbo_gnn g, const rbo_csr* A, const double* R, int32_t nr, int64_t ldr,
                       float lr, double* loss, void* stream) {
  if (!g || !R || nr < 1 || nr > 64 || !loss || !(lr > 0.f)) return RBO_ERR_ARG;
  int e = check_csr(A);
  if (e) return e;
  if (ldr < A->n) return RBO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  Arena* ar = nullptr;
  int launches = 0;
  if ((e = loss_grad(g, A, R, nr, ldr, loss, &ar, st, &launches))) return e;
  g->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)g->step), c2 = 1.f - std::pow(b2, (float)g->step);
  adam_kernel<<<grid1(NPARAM), 256, 0, st>>>(NPARAM, g->theta, g->grad, g->m1, g->m2, lr, b1, b2,
                                             1e-8f, c1, c2, g->wbf);
  if ((e = note_cuda(cudaGetLastError()))) return e;
  return finish_status(ar, st, nullptr);
}

}  // extern "C"

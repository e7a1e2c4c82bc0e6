// One-CTA small dense kernels run by the last CTA of a row pass (data in shared
// memory, all NT threads cooperating): upper Cholesky with breakdown detection,
// Householder QR with non-negative diagonal (R and thin Q), and the sketched
// BCGS2 with Householder intra step of the two-stage preprocessing.
#pragma once

#include "device_common.cuh"

namespace rbo {

// In-place upper Cholesky of the b x b symmetric matrix G (column-major, ld b, only
// the upper triangle is read).  On exit the upper triangle holds R (G = R^T R) and
// the strict lower triangle is zeroed.  Returns -1, or the first column whose pivot
// is not positive / not finite (Section 5.1: "non-positive pivots").
static __device__ int cta_cholesky(double* G, int b, int* s_flag) {
  const int tid = threadIdx.x;
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      double piv = G[j + j * b];
      for (int i = 0; i < j; ++i) piv -= G[i + j * b] * G[i + j * b];
      if (!(piv > 0.0) || !isfinite(piv)) {
        *s_flag = j;
      } else {
        G[j + j * b] = sqrt(piv);
        *s_flag = -1;
      }
    }
    __syncthreads();
    const int bad = *s_flag;
    __syncthreads();
    if (bad >= 0) return bad;
    const double inv = 1.0 / G[j + j * b];
    for (int c = j + 1 + tid; c < b; c += blockDim.x) {
      double v = G[j + c * b];
      for (int i = 0; i < j; ++i) v -= G[i + j * b] * G[i + c * b];
      G[j + c * b] = v * inv;
    }
    __syncthreads();
  }
  for (int e = tid; e < b * b; e += blockDim.x) {
    int i = e % b, c = e / b;
    if (i > c) G[e] = 0.0;
  }
  __syncthreads();
  return -1;
}

// First column j whose diagonal entry R_jj of the k x k triangular factor (ld k) is
// not finite or within k * 2^-53 of the largest |R_ii|: the factored block is rank
// deficient to working precision.  -1 if none.  Call from one thread.
__device__ inline int tri_rank_deficient(const double* R, int k) {
  double rmax = 0.0;
  for (int j = 0; j < k; ++j) {
    const double v = fabs(R[j + j * k]);
    if (!(v <= 1.7976931348623157e308)) return j;  // NaN or infinity
    rmax = fmax(rmax, v);
  }
  const double tol = (double)k * 0x1p-53 * rmax;
  for (int j = 0; j < k; ++j)
    if (!(fabs(R[j + j * k]) > tol)) return j;
  return -1;
}

// Householder QR of A (m x k, column-major ld m) in shared memory.  On exit
// R (k x k, ld k) holds the triangular factor with a non-negative diagonal; if Q
// is non-null it receives the thin orthogonal factor (m x k, ld m) with the same
// column signs.  A is overwritten by the reflectors.  `beta` needs k doubles,
// `sgn` k doubles; `red` (32 doubles) is not used.
static __device__ void cta_householder(double* A, int m, int k, double* R, double* Q, double* beta,
                                double* sgn, double* red) {
  // Sequential float64 latency, not throughput, bounds this on one SM: the norm and the
  // reflector of each column are formed by warp 0 alone (one warp reduction, one square
  // root and division by lane 0), the updates of the columns to the right by one warp
  // each, and every column of Q by its own warp without block barriers.
  (void)red;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < k * k; e += blockDim.x) R[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    double* a = A + (size_t)j * m;
    if (warp == 0) {
      double p0 = 0.0, p1 = 0.0;
      int i = j + 1 + lane;
      for (; i + 32 < m; i += 64) {
        p0 = fma(a[i], a[i], p0);
        p1 = fma(a[i + 32], a[i + 32], p1);
      }
      if (i < m) p0 = fma(a[i], a[i], p0);
      const double rest = warp_sum(p0 + p1);
      if (lane == 0) {
        const double x0 = a[j];
        const double alpha = sqrt(rest + x0 * x0);
        const double s = x0 >= 0.0 ? 1.0 : -1.0;
        const double v0 = x0 + s * alpha;
        const double vtv = rest + v0 * v0;
        a[j] = v0;
        beta[j] = (alpha == 0.0) ? 0.0 : 2.0 / vtv;
        R[j + j * k] = -s * alpha;
      }
    }
    __syncthreads();
    const double bj = beta[j];
    // apply H_j = I - bj v v^T to the columns to the right (one warp per column)
    for (int c = j + 1 + warp; c < k; c += nw) {
      double* ac = A + (size_t)c * m;
      double w = 0.0;
      for (int i = j + lane; i < m; i += 32) w += a[i] * ac[i];
      w = warp_sum(w) * bj;
      for (int i = j + lane; i < m; i += 32) ac[i] -= w * a[i];
      __syncwarp();
      if (lane == 0) R[j + c * k] = ac[j];
    }
    __syncthreads();
  }
  // sign fix: diag(R) >= 0
  for (int j = tid; j < k; j += blockDim.x) sgn[j] = R[j + j * k] < 0.0 ? -1.0 : 1.0;
  __syncthreads();
  for (int e = tid; e < k * k; e += blockDim.x) {
    int i = e % k;
    R[e] *= sgn[i];
  }
  if (Q != nullptr) {
    // Q = H_0 ... H_{k-1} [I; 0]: column c is H_0 ... H_c e_c (H_j e_c = e_c for
    // j > c, the reflector of column j being zero above row j), one warp per column
    for (int c = warp; c < k; c += nw) {
      double* qc = Q + (size_t)c * m;
      for (int i = lane; i < m; i += 32) qc[i] = (i == c) ? 1.0 : 0.0;
      __syncwarp();
      for (int j = c; j >= 0; --j) {
        const double* a = A + (size_t)j * m;
        double w = 0.0;
        for (int i = j + lane; i < m; i += 32) w += a[i] * qc[i];
        w = warp_sum(w) * beta[j];
        for (int i = j + lane; i < m; i += 32) qc[i] -= w * a[i];
        __syncwarp();
      }
      for (int i = lane; i < m; i += 32) qc[i] *= sgn[c];
    }
  }
  __syncthreads();
}

// C (p x k, ld p) = Qs^T V for Qs (m x p, ld ldq, global) and V (m x k, ld m, shared).
// Each dot product is split over S consecutive lanes of a warp (S the largest power of
// two with p k S <= threads), two interleaved chains per lane, then summed by lane
// shuffles: the float64 work spreads over every thread while the dependent chains
// stay short (the float64 pipe of this GPU does 2 lane-FMAs per SM and cycle).
static __device__ void cta_gemm_tn(const double* Qs, int ldq, const double* V, int m, int p, int k,
                                   double* C) {
  const int nout = p * k;
  int S = 32;
  while (S > 1 && nout * S > (int)blockDim.x) S >>= 1;
  const int per = (int)blockDim.x / S;
  for (int e0 = 0; e0 < nout; e0 += per) {
    const int e = e0 + (int)threadIdx.x / S, sl = (int)threadIdx.x % S;
    double s0 = 0.0, s1 = 0.0;
    if (e < nout) {
      const double* q = Qs + (size_t)(e % p) * ldq;
      const double* v = V + (size_t)(e / p) * m;
      int r = sl;
      for (; r + S < m; r += 2 * S) {
        s0 = fma(q[r], v[r], s0);
        s1 = fma(q[r + S], v[r + S], s1);
      }
      if (r < m) s0 = fma(q[r], v[r], s0);
    }
    double s = s0 + s1;
    for (int o = S >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (e < nout && sl == 0) C[e] = s;
  }
  __syncthreads();
}

// V (m x k, ld m, shared) -= Qs (m x p, global) C (p x k, ld p), one entry per task
static __device__ void cta_gemm_nn_sub(const double* Qs, int ldq, const double* C, int m, int p, int k,
                                       double* V) {
  for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
    int r = e % m, c = e / m;
    double s = V[e];
    for (int i = 0; i < p; ++i) s -= Qs[(size_t)i * ldq + r] * C[i + c * p];
    V[e] = s;
  }
  __syncthreads();
}

// Bring the p columns of Qs (m x p, ld ldq, global) into this SM's L1 before the
// small products read them (one 128-byte line per thread and step).
static __device__ void cta_prefetch_cols(const double* Qs, int ldq, int m, int p) {
  const int lines = (m * 8 + 127) / 128;
  for (int t = threadIdx.x; t < lines * p; t += blockDim.x) {
    const double* a = Qs + (size_t)(t / lines) * ldq + (size_t)(t % lines) * 16;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
  }
}

}  // namespace rbo

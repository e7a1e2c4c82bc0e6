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
// `sgn` k doubles, `red` 32 doubles.
static __device__ void cta_householder(double* A, int m, int k, double* R, double* Q, double* beta,
                                double* sgn, double* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < k * k; e += blockDim.x) R[e] = 0.0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    double* a = A + (size_t)j * m;
    double part = 0.0;
    for (int i = j + 1 + tid; i < m; i += blockDim.x) part += a[i] * a[i];
    const double rest = block_sum(part, red);
    const double x0 = a[j];
    const double alpha = sqrt(rest + x0 * x0);
    const double s = x0 >= 0.0 ? 1.0 : -1.0;
    const double v0 = x0 + s * alpha;
    const double vtv = rest + v0 * v0;
    const double bj = (alpha == 0.0) ? 0.0 : 2.0 / vtv;
    __syncthreads();
    if (tid == 0) {
      a[j] = v0;
      beta[j] = bj;
      R[j + j * k] = -s * alpha;
    }
    __syncthreads();
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
    // Q = H_0 ... H_{k-1} [I; 0], accumulated backwards, one warp per column
    for (int e = tid; e < m * k; e += blockDim.x) {
      int i = e % m, c = e / m;
      Q[e] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = k - 1; j >= 0; --j) {
      const double* a = A + (size_t)j * m;
      const double bj = beta[j];
      for (int c = warp; c < k; c += nw) {
        double* qc = Q + (size_t)c * m;
        double w = 0.0;
        for (int i = j + lane; i < m; i += 32) w += a[i] * qc[i];
        w = warp_sum(w) * bj;
        for (int i = j + lane; i < m; i += 32) qc[i] -= w * a[i];
      }
      __syncthreads();
    }
    for (int e = tid; e < m * k; e += blockDim.x) Q[e] *= sgn[e / m];
  }
  __syncthreads();
}

// C (p x k, ld p) = Qs^T V for Qs (m x p, ld ldq, global) and V (m x k, ld m, shared):
// one warp per (i, c) dot product.
static __device__ void cta_gemm_tn(const double* Qs, int ldq, const double* V, int m, int p, int k,
                            double* C) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int e = warp; e < p * k; e += nw) {
    int i = e % p, c = e / p;
    const double* q = Qs + (size_t)i * ldq;
    const double* v = V + (size_t)c * m;
    double s = 0.0;
    for (int r = lane; r < m; r += 32) s += q[r] * v[r];
    s = warp_sum(s);
    if (lane == 0) C[e] = s;
  }
  __syncthreads();
}

// V (m x k, ld m, shared) -= Qs (m x p, global) C (p x k, ld p)
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

}  // namespace rbo

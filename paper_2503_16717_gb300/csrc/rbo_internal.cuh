// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/rbo.h"

// The sketch handle of the C ABI: parameters only, entries are recomputed.
struct rbo_sketch_s {
  int64_t n_max;
  int32_t d;        // rows of the sketch S W
  int32_t zeta;     // sparse-sign: nonzeros per column (Count-Gauss: 1, in the Count stage)
  uint64_t seed;
  int32_t type = 0;     // RBO_SKETCH_*
  int32_t d_inner = 0;  // Count-Gauss: rows of the Count stage
};

namespace rbo {

// Largest d * k (sketch rows x panel columns): the per-warp sketch partials of a row
// pass live in shared memory.
constexpr int64_t MAX_SKETCH_DK = 12288;

// The sketch's shared-memory and Z-row limits for panels of up to kmax columns.
inline bool sketch_fits(const ::rbo_sketch_s* sk, int kmax) {
  switch (sk->type) {
    case RBO_SKETCH_GAUSSIAN: return sk->d * kmax <= 8192;
    case RBO_SKETCH_COUNT_GAUSS:
      return (int64_t)sk->d_inner * kmax <= MAX_SKETCH_DK && (int64_t)sk->d * kmax <= MAX_SKETCH_DK;
    default: return (int64_t)sk->d * kmax <= MAX_SKETCH_DK;
  }
}


// Static scratch of rbo_gram_noalloc (see include/rbo.h).
#define RBO_NOALLOC_SCRATCH_BYTES (4u << 20)
#define RBO_NOALLOC_MAX_AB 2048

// ---- device status word -----------------------------------------------------------
// Every kernel reads `code` first and returns at once when an earlier kernel of the
// same call failed, so one host read at the end of a call reports the first failure.
struct DevStatus {
  int code;     // 0 or an RBO_ERR_* value
  int block;    // block / big-panel index of a Cholesky breakdown
  int column;   // column of the failed pivot within that block
  int stage;    // RBO_STAGE_*
  int where;    // kernel tag for timeouts
  int pad[3];
};

// ---- per-device workspace arena -----------------------------------------------------
struct Arena {
  int device = -1;
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  DevStatus* status = nullptr;   // device, first 256 bytes of the arena
  DevStatus* status_host = nullptr;  // pinned host mirror
  unsigned* tickets = nullptr;   // device, n_tickets counters (bytes 64..255)
  int n_tickets = 0;
  double* red = nullptr;         // cross-CTA reduction scratch of the current call
  size_t red_bytes = 0;
  void reset() { used = 256; red = nullptr; red_bytes = 0; }
  // bump allocation, 256-byte aligned; returns nullptr when `cap` is too small
  void* take(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    if (off + bytes > cap) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

// Grow (if needed) and reset the arena of the current device so that at least
// `bytes` are available after the status block.  Returns RBO_OK or an error.
int arena_prepare(Arena** out, size_t bytes);
// Carve the reduction scratch (partials + group partials) for a call whose passes
// have at most `max_L` reduced values, and zero the tickets.  Call right after
// arena_prepare, before other takes.
int arena_reserve_reduction(Arena* ar, int max_L, cudaStream_t st);
// Bytes arena_reserve_reduction will take for `max_L`.
size_t reduction_bytes(int max_L);
int arena_release_current();

// ---- the row-pass kernel (tall-skinny fused pass) ---------------------------------
enum EpiOp : int {
  EPI_NONE = 0,
  EPI_STORE = 1,      // write the reduced X^T Y' block to out (ld out_ld, offsets)
  EPI_CHOL = 2,       // Cholesky of the reduced Y'^T Y' -> out_r (b x b, ld b)
  EPI_HH = 3,         // Householder R of the reduced sketch -> out_r
  EPI_SKB2 = 4,       // two-stage: sketched BCGS2-HH against the stored sketched basis
  EPI_GB = 5,         // two-stage: store [X Y']^T Y' as block column of G_B; Cholesky at end
  EPI_STORE_ALL = 6,  // write all of Z (zr x b, ld zr) to out and the sketch (d x b) to out_sk
  EPI_PIP = 7,        // two-stage BCGS-PIP: Z = [Qbar_{<j} Vh]^T Vh; T_jj = chol(G - P^T P);
                      // T(0:poff, poff:poff+b) = P, T(poff:, poff:) = T_jj
  EPI_SKETCH_OUT = 8, // write the sketch S Y' (rows x b, column-major) to out_sk
};

enum AssembleOp : int {
  ASM_NONE = 0,
  ASM_ONE_STAGE = 1,  // R_top = C1 + C2 (R' Rh), R_jj = R2 R' Rh
  ASM_TWO_STAGE = 2,  // R_QB = C1 + C2 R' T, R_BB = R2 R' T, coords = [C2 R'; R2 R']
  ASM_DIAG = 3,       // R_jj = R2 (single normalisation)
};

struct Epilogue {
  int op = EPI_NONE;
  // EPI_STORE: Z rows [0, a) go to out[(row_off + i) + (col_off + c) * out_ld]
  double* out = nullptr;
  int out_ld = 0, row_off = 0, col_off = 0;
  double* out_sk = nullptr;
  // EPI_CHOL / EPI_HH: R (b x b, ld b)
  double* out_r = nullptr;
  int stage = 0, block = 0;
  // EPI_SKB2: sketched basis qs (d x K, ld d), T (K x K, ld K), current offset p'
  double* qs = nullptr;
  double* T = nullptr;
  int K = 0, poff = 0;
  // EPI_GB: G_B (K x K, ld K) block column at poff; chol of G_B when `last`
  double* GB = nullptr;
  int last = 0;
  double* out_rp = nullptr;  // R' (K x K, ld K)
  // assembly after a Cholesky (all device, column-major)
  int asm_op = ASM_NONE;
  const double* C1 = nullptr; int ldc1 = 0;   // p x k (or P x K)
  const double* C2 = nullptr; int ldc2 = 0;   // p x k
  const double* Rh = nullptr;                 // k x k (R_hat or T)
  const double* Rp = nullptr;                 // k x k (R')
  double* Rfull = nullptr; int ldR = 0;       // ncols x ncols result
  int p = 0, col0 = 0;                        // rows above, first column of the block
  double* coords = nullptr; int ldcoords = 0; // two-stage: (p + k) x k coordinates of Qbar
};

struct SketchSched {
  const uint8_t* rec = nullptr;  // ceil(n / T) records of rec_bytes
  int T = 0, mcap = 0, rec_bytes = 0;
};

struct RowPass {
  int64_t n = 0;
  const double* X = nullptr; int64_t ldx = 0; int a = 0;
  double* Y = nullptr; int64_t ldy = 0; int b = 0;
  const double* C = nullptr;     // a x b (ld ldc): projection coefficients, null = none
  int ldc = 0;                   // 0 means a
  const double* Tri = nullptr;   // b x b (ld ldtri) upper triangular, null = none
  int ldtri = 0;                 // 0 means b
  int tri_first = 0;             // 1: y' = y Tri^-1 - x C;  0: y' = (y - x C) Tri^-1
  int write_y = 0;
  int acc_x = 0;                 // accumulate X^T Y'
  int acc_y = 0;                 // accumulate Y'^T Y'
  int sk_d = 0, sk_zeta = 0; uint64_t sk_seed = 0;  // accumulate S Y' (d x b), sparse-sign
  SketchSched sk;                // sketch schedule of the n rows (required with sk_d > 0)
  int sk_gd = 0;                 // Gaussian sketch rows (entries generated per tile; Z rows)
  int sk_cg = 0;                 // Count-Gauss: final rows (Gaussian stage in the epilogue;
                                 // sk_d is then the Count stage, zeta 1)
  int mixed = 0;                 // float32 accumulation of X^T Y' and S Y'
  int df64 = 0;                  // float32-pair arithmetic for the Gram (and small projections)
  int ozaki = 0;                 // Gram on the tensor cores (exact digit products, ozaki.cu):
                                 // 1 where the pass shape allows it and it is the faster
                                 // kernel, 2 wherever the shape allows it; float64 otherwise
  int small_coeffs = 0;          // C is a re-orthogonalization (O(eps kappa)) coefficient block
  int max_ctas = 0;              // cap on the grid (0: none); bounds the reduction scratch
  int tag = 0;                   // role for the per-kernel timing (RBO_PROF_PASS_*)
  Epilogue epi;
};

// Tensor-core Gram pass (ozaki.cu): whether it serves `rp` (rp.ozaki set, a Gram of at most
// 64 A columns and 8 Y' columns, no projection and no sketch), and its launcher.
bool ozaki_gram_supported(const RowPass& rp);
// Whether the digit-product kernel beats the float64 pass for this shape: its time per
// row is nearly flat in the column count (the digit formation and the tensor-core
// handshakes per 16-row step dominate), the float64 pass's grows with a * b.
bool ozaki_gram_pays(const RowPass& rp);
int ozaki_gram_launch(const RowPass& rp, Arena* ar, cudaStream_t st, int* launches, int num_sms);

// Enqueue one row pass; `launches` is incremented per kernel.  Returns RBO_OK or an
// error for invalid sizes / CUDA launch failures.
int rowpass_launch(const RowPass& rp, Arena* ar, cudaStream_t st, int* launches);
// The sketch-scatter pass (rowpass_sk.cu), called by rowpass_launch for a pass with a
// scattered sketch once the common checks passed: `L` partial length (d * b), `mixed`
// float32 sketch sums.
int rowpass_sk_launch(const RowPass& rp, Arena* ar, cudaStream_t st, int* launches, int num_sms,
                      int L, int mixed);
// Shared-memory bytes of its streaming loop for a X columns, b panel columns, T-row
// tiles and a d-row, zeta-entry sparse sketch (with a projection and a triangle).
size_t rowpass_sk_loop_bytes(int a, int b, int T, int d, int zeta);

// Sketch schedule: S restricted to each tile of T basis rows, transposed once per
// call so that the row pass needs neither hashing nor a scatter with conflicts.
// Record of a tile (rec_bytes, a 16-byte multiple):
//   meta[mcap] (uint32): one per non-empty sketch row i of the tile, sorted by the
//       number of entries (descending, then i): i | offset << 12 | count << 23;
//       0xFFFFFFFF past the last;
//   list[T * zeta] (uint8): the tile's entries grouped by sketch row (rows in
//       increasing order within a group): local row << 1 | (sign < 0).
int sketch_sched_mcap(int T, int d, int zeta);
int sketch_sched_rec_bytes(int T, int d, int zeta);
size_t sketch_sched_bytes(int64_t n, int T, int d, int zeta);
// Builds the records of all ceil(n / T) tiles into `out` (sketch_sched_bytes).
int sketch_sched_launch(int64_t n, int T, int d, int zeta, uint64_t seed, uint8_t* out,
                        DevStatus* status, cudaStream_t st);
// Tile height (128, 64, 32 or 16) that every sketch pass with at most a_max X columns and
// b_max panel columns can use (the schedule is built for it).
int rowpass_sketch_T(int a_max, int b_max, int d, int zeta);

// Sketch entries materialisation and a standalone sketch apply (entry points).
int sketch_entries_launch(int64_t row0, int64_t nrows, int d, int zeta, uint64_t seed,
                          int32_t* idx, int8_t* sign, DevStatus* status, cudaStream_t st);

// ---- sparse kernels ------------------------------------------------------------------
struct CsrDev {
  int64_t n, nnz;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
};
// Optional epilogue of an SpMV: y = (A x) + a u + b uprev (u null: none; uprev null or
// b == 0: no third term), with the arithmetic of the separate shift pass (two fmas).
struct SpmvShift {
  const double* u = nullptr;
  double a = 0.0;
  const double* uprev = nullptr;
  double b = 0.0;
};
// y = A (D x) (D = diag(dscale) when dscale != null), then the optional shift
// Invalid indices are skipped and reported in `status` (may be null).
int spmv_launch(const CsrDev& A, const double* dscale, const double* x, double* y,
                DevStatus* status, cudaStream_t st, const SpmvShift& sh = SpmvShift());
// Sliced ELL copy of a CSR matrix with short rows (SELL-32): slices of 32 consecutive
// rows, each slice padded to its longest row; slot j of row 32 k + l at
// soff[k] + 32 j + l, padding slots hold the row's own index and the value 0.
struct SellDev {
  int64_t n = 0, nslices = 0;    // n = 0: not built
  const int64_t* soff = nullptr; // nslices + 1 slot offsets
  const int32_t* col = nullptr;
  const double* val = nullptr;
};
// Slots needed by the SELL-32 copy of A if its padding stays within `cap_slots`:
// builds it into (soff, col, val) and fills *out, else leaves out->n = 0.  Column
// indices outside [0, n) and malformed row pointers are reported in `status` (and
// stored as zero entries).  One host synchronisation (the slice widths).
int sell_build(const CsrDev& A, int64_t cap_slots, int64_t* soff, int32_t* width_scratch, int32_t* col,
               double* val, DevStatus* status, cudaStream_t st, SellDev* out);
// y = A x with the optional shift, from the SELL-32 copy
int spmv_sell_launch(const SellDev& S, int64_t nnz, const double* x, double* y, cudaStream_t st,
                     const SpmvShift& sh = SpmvShift());
// r = b - A x  (A already scaled if needed)
int residual_launch(const CsrDev& A, const double* b, const double* x, double* r, DevStatus* status,
                    cudaStream_t st);
// val_out[j] = val[j] * dscale[col[j]]
int scale_columns_launch(const CsrDev& A, const double* dscale, double* val_out, cudaStream_t st);
// dscale[i] = 1 / A[i][i]; status error when a diagonal entry is zero or missing
int jacobi_launch(const CsrDev& A, double* dscale, DevStatus* status, cudaStream_t st);
// y = Q z (accumulate 0) or y += Q z  (Q n x k, ld ldq; z device k)
int gemv_update_launch(int64_t n, int k, const double* Q, int64_t ldq, const double* z, double* y,
                       int accumulate, cudaStream_t st);
// x += diag(ds) t  (ds null: x += t)
int axpy_scaled_launch(int64_t n, const double* ds, const double* t, double* x, cudaStream_t st);
// mode 0: x = dscale .* y;  mode 1: x = y ./ dscale  (dscale null: copy)
int scale_vec_launch(int64_t n, const double* dscale, const double* y, double* x, int mode,
                     cudaStream_t st);

// ---- host orchestration ----------------------------------------------------------------
struct OrthCtx {
  Arena* ar = nullptr;
  cudaStream_t st = nullptr;
  int launches = 0;
  int mixed = 0;
  int df64 = 0;   // every pass in float32-pair arithmetic where it applies
  int ozaki = 0;  // Gram passes on the tensor cores where the pass shape allows
  int d = 0, zeta = 0; uint64_t seed = 0;  // d: rows of the (final) sketch
  int sk_type = 0, d_inner = 0;            // RBO_SKETCH_*; Count-Gauss Count-stage rows
  int pip = 0;      // two-stage preprocessing by BCGS-PIP instead of RandBCGS2
  SketchSched sk;   // sketch schedule of the call's n rows
  // small device buffers, sized once per call by orth_ctx_alloc and reused by every
  // block (stream order makes the reuse safe)
  int pmax = 0, kmax = 0;
  double *C1 = nullptr, *C2 = nullptr, *Rh = nullptr, *Rp = nullptr, *R2 = nullptr;
  double *T = nullptr, *qs = nullptr, *GB = nullptr;
  double* tmp = nullptr;  // pmax*kmax + kmax*kmax doubles for small staging
};
// Take the small buffers from the arena for blocks with up to pmax previous columns
// and kmax columns per block (K for two-stage).  Returns RBO_OK or RBO_ERR_NOMEM.
// With a sketch (c.d > 0) it also builds the sketch entry table of n rows.
int orth_ctx_alloc(OrthCtx& c, int pmax, int kmax, int64_t n);
// Arena bytes orth_ctx_alloc will need.
// (d: rows of the final sketch; type RBO_SKETCH_*; d_inner: Count-Gauss Count stage)
size_t orth_ctx_bytes(int pmax, int kmax, int d, int64_t n, int zeta, int type, int d_inner);
// Newton-basis shifts from the k x k upper Hessenberg H (ld ld): alpha, beta (s each).
int newton_shifts(const double* H, int64_t ld, int k, int s, double* alpha, double* beta);
int chebyshev_shifts(const double* H, int64_t ld, int k, int s, double* alpha, double* beta);
// Sketch fields of a row pass that applies the call's sketch.
void set_sketch(RowPass& r, const OrthCtx& c);
// Largest reduced-vector length of any pass for these sizes.
int orth_max_L(int pmax, int kmax, int d);

// One-stage BCGS2 of the k columns W (ld ldw) against Q (p columns, ld ldq): on exit W
// holds Q_j.  Block index `blk` for breakdown reports.  R block (rows 0..p+k-1, cols
// col0..col0+k-1) is written to Rdev (ld ldR).  intra: RBO_INTRA_*.
int one_stage_block(OrthCtx& c, int64_t n, const double* Q, int64_t ldq, int p, double* W,
                    int64_t ldw, int k, int intra, double* Rdev, int ldR, int col0, int blk);

// Normalise one column (V_0): R[col0][col0] = ||v||.
int normalise_column(OrthCtx& c, int64_t n, double* v, double* Rdev, int ldR, int col0);

// Two-stage big panel processing, panel by panel (used by the flat scheme and GMRES).
struct BigPanel {
  int64_t n = 0;
  const double* Q = nullptr; int64_t ldq = 0; int P = 0;   // finished basis
  double* VB = nullptr; int64_t ldv = 0;                   // big panel columns (K)
  int K = 0;                                               // s_hat
  int cols = 0;                                            // columns preprocessed so far
  int blk = 0;                                             // big panel index
};
// Preprocess panel of k columns stored at VB + cols*ldv (in place -> Qbar_j).
int bigpanel_add(OrthCtx& c, BigPanel& bp, int k);
// Finish: VB holds Q_B; R written at rows 0..P+K-1, cols col0..; coords (P+K) x K of Qbar.
int bigpanel_finish(OrthCtx& c, BigPanel& bp, double* Rdev, int ldR, int col0, double* coords,
                    int ldcoords);

// Read the device status (synchronises the stream) and fill info's breakdown fields.
int finish_status(Arena* ar, cudaStream_t st, rbo_info* info);

// Record a CUDA error for rbo_last_error(); returns RBO_OK for cudaSuccess, else
// RBO_ERR_CUDA.
int note_cuda(cudaError_t e);

// ---- optional per-kernel timing (rbo_profile_*) ----------------------------------------
// kinds 0..7: RBO_PROF_*; 8 + tag: row passes by role (RowPass::tag)
constexpr int PROF_KINDS = 32;
struct ProfToken {
  void* ev = nullptr;
};
bool prof_on();
ProfToken prof_start(cudaStream_t st);
void prof_stop(const ProfToken& t, cudaStream_t st, int kind, double bytes, double flops,
               int tag = -1);
void prof_drain();

}  // namespace rbo

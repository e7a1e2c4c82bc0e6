/*
 * rbo.h -- randomized block orthogonalization for s-step GMRES on GB300 (sm_103a).
 *
 * C ABI of the library librbo.so.  The operations follow Yamazaki, Higgins,
 * Boman and Szyld, "Random sketching to enhance the numerical stability of
 * block orthogonalization algorithms for s-step GMRES" (arXiv 2503.16717):
 *
 *   qr(Q, V_j):  extend Q R = V with Q^T Q = I, R upper triangular with a
 *                non-negative diagonal (Section 4, Figure 1 caption).
 *
 * Conventions shared by every call
 *   - Dense n-row arrays (V, Q, vectors) are caller-owned DEVICE pointers,
 *     column-major with leading dimension ld >= n, float64.
 *   - Small outputs (R, info) are caller-owned HOST memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on that stream; every call that returns a
 *     status synchronises the stream once at its end to read the device
 *     status word (and GMRES synchronises once per panel for its host-side
 *     least-squares step).
 *   - Scratch memory comes from a per-device library arena that grows on
 *     demand (cudaMalloc) and is reused by later calls; rbo_release_workspace
 *     frees it.  Calls that share the arena must not overlap in time (use one
 *     host thread / one stream per device at a time).
 *   - Every call returns RBO_OK (0) or a negative RBO_ERR_* code; no call
 *     throws or aborts.  On an error the contents of the in/out arrays are
 *     unspecified.
 *   - The library caches per-device state (the workspace arena, launch facts,
 *     device addresses of static arrays); it must not be used on a device across
 *     a cudaDeviceReset of that device.
 */
#ifndef RBO_H
#define RBO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define RBO_OK                  0
#define RBO_ERR_ARG            -1  /* invalid argument (size, pointer, layout)          */
#define RBO_ERR_CUDA           -2  /* a CUDA runtime call failed                         */
#define RBO_ERR_CHOL_BREAKDOWN -3  /* non-positive Cholesky pivot (Section 5.1);
                                      info->breakdown_* say where                        */
#define RBO_ERR_NOT_CONVERGED  -4  /* GMRES reached max_restarts above tol               */
#define RBO_ERR_TIMEOUT        -5  /* a bounded device wait expired                      */
#define RBO_ERR_SKETCH         -6  /* a sketch column found < zeta distinct rows         */
#define RBO_ERR_NOMEM          -7  /* workspace allocation failed                        */
#define RBO_ERR_NO_DEVICE      -8  /* no CUDA device / not an sm_103 device              */
#define RBO_ERR_LOST_ORTHOGONALITY -9  /* the final CholQR of a block met a Gram far from I:
                                      the first intra-block step failed at the working
                                      precision (block numerically rank deficient, or
                                      beyond the mixed-precision range); info->
                                      breakdown_block says which block                   */

/* ---- precision modes --------------------------------------------------------- */
#define RBO_PREC_FP64   0  /* every step in IEEE float64 (the reference path)          */
#define RBO_PREC_MIXED  1  /* sketch apply and first-pass projection coefficients in
                              float32 with float32 accumulation; Gram matrices feeding
                              the final Cholesky, the small factors, every update of V
                              and the final TRSM in float64                             */
#define RBO_PREC_DF64   2  /* float64 data; every Gram matrix and the re-orthogonalization
                              update (whose coefficients are O(eps kappa)) in float32
                              pairs (about 48 significant bits, error-free
                              transformations on the FP32 pipe, Gram sums flushed to
                              float64 every ~64 terms); first-pass projections, TRSMs,
                              the sketch and the small factors in float64.  Only steps
                              that cannot reach the backward error ||V - QR|| are
                              moved off the float64 pipe                              */
#define RBO_PREC_OZAKI  3  /* float64 data and results; the wide Gram matrices of the BCGS
                              and CholQR reductions (passes of 36 to 64 columns of [X Y'],
                              at most 8 of Y', no projection, no triangular solve) are
                              computed on the fp16 tensor cores from exact integer
                              products: per accumulation chunk of up to 1024 rows every
                              value is scaled by a power of two of its column to an
                              integer below 2^53, split into 7 balanced 8-bit digits
                              (each exact in fp16), the digit products are summed
                              exactly in float32 and the pairs of digit levels
                              I + J <= 7 are combined in 64/128-bit integers (Ozaki,
                              Ogita, Oishi and Rump 2012); every other pass as
                              RBO_PREC_FP64                                           */

/* ---- intra-block choice (one-stage) ----------------------------------------- */
#define RBO_INTRA_RANDCHOLQR 0  /* RandCholQR (Figure 4b)                                */
#define RBO_INTRA_CHOLQR2    1  /* CholQR2 (Figure 2b twice): the deterministic baseline */

typedef struct rbo_opts {
  int32_t precision;     /* RBO_PREC_*                                                  */
  int32_t v0;            /* 1: column 0 of V is the single start vector V_0 = [v_0]
                            (Table 1), normalised before the blocks                     */
  int32_t intra;         /* RBO_INTRA_*: one-stage only (block_orth_one_stage and the
                            one-stage s-step GMRES); RBO_ERR_ARG for CHOLQR2 with s_hat > s */
  int32_t max_restarts;  /* GMRES: restart cycles allowed (default 1000 if <= 0)        */
  int32_t precond;       /* GMRES: 0 none, 1 Jacobi (M = diag(A), right preconditioner) */
  int32_t preproc;       /* two-stage: RBO_PREPROC_* (0 = RandBCGS2)                   */
  int32_t basis;         /* GMRES: RBO_BASIS_* (0 = monomial)                           */
  int32_t reserved[1];
} rbo_opts;

#define RBO_STAGE_V0          1  /* normalisation of v_0                                  */
#define RBO_STAGE_INTRA       2  /* first intra-block Cholesky (CholQR / RandCholQR)     */
#define RBO_STAGE_INTRA2      3  /* second Cholesky of CholQR2                           */
#define RBO_STAGE_FINAL       4  /* Cholesky after the re-orthogonalization              */
#define RBO_STAGE_BIGPANEL    5  /* two-stage: CholQR of the preprocessed big panel      */
#define RBO_STAGE_PREPROC     6  /* two-stage BCGS-PIP: Cholesky of the Pythagorean Gram */

/* sketch types (rbo_sketch_create_ex; Section 5.2) */
#define RBO_SKETCH_SPARSE_SIGN 0  /* zeta +-1 per column (zeta = 1: the Count sketch)     */
#define RBO_SKETCH_GAUSSIAN    1  /* dense N(0, 1) entries, generated from the seed        */
#define RBO_SKETCH_COUNT_GAUSS 2  /* Count sketch to d_inner rows, then a d x d_inner
                                     Gaussian map                                        */

/* matrix-powers basis of s-step GMRES (rbo_opts.basis) */
#define RBO_BASIS_MONOMIAL    0  /* v_{i+1} = A M v_i (the paper's choice)                */
#define RBO_BASIS_NEWTON      1  /* first cycle standard GMRES, then Newton steps with the
                                    Leja-ordered Ritz values of the first cycle's
                                    Hessenberg matrix as shifts (rbo_newton_shifts)      */
#define RBO_BASIS_CHEBYSHEV   2  /* first cycle standard GMRES, then the Chebyshev basis
                                    of the ellipse enclosing its Ritz values
                                    (rbo_chebyshev_shifts)                               */

/* two-stage preprocessing of the panels of a big panel (rbo_opts.preproc) */
#define RBO_PREPROC_RAND      0  /* RandBCGS2: sketch + sketched BCGS2-HH (Section 7.2)  */
#define RBO_PREPROC_PIP       1  /* BCGS-PIP: one reduction of [Qbar V]^T V, Cholesky of
                                    G - P^T P (Section 7.1); no sketch                   */

typedef struct rbo_info {
  int32_t status;            /* same value as the return code                          */
  int32_t breakdown_block;   /* block (one-stage) or big panel (two-stage), -1 if none */
  int32_t breakdown_column;  /* column within that block of the failed pivot           */
  int32_t breakdown_stage;   /* RBO_STAGE_*                                            */
  int32_t iterations;        /* GMRES: matrix-powers columns generated                */
  int32_t restarts;          /* GMRES: restart cycles started                          */
  int32_t converged;         /* GMRES: 1 if ||b - A x|| <= tol ||b||                    */
  int32_t kernel_launches;   /* kernels this call enqueued                              */
  double  relres;            /* GMRES: final true relative residual                    */
  double  est_relres;        /* GMRES: last least-squares residual estimate            */
  double  time_ms;           /* host wall time of the call                             */
  double* history;           /* GMRES, optional caller buffer: (iteration, true relres)
                                pairs, one per restart                                 */
  int32_t history_cap;       /* capacity of `history` in pairs                         */
  int32_t history_len;       /* pairs written                                          */
  double* resid;             /* GMRES, optional caller DEVICE buffer (n x resid_cap,
                                ld resid_ld): the true residual b - A x at the start
                                of each restart cycle (training data for the learned
                                preconditioner)                                        */
  int64_t resid_ld;
  int32_t resid_cap;
  int32_t resid_len;         /* residual columns written                              */
  int32_t fallbacks;         /* RBO_PREC_MIXED: GMRES restart cycles, or blocks (two-stage:
                                big panels) of a block orthogonalization, redone in
                                float64 after a block lost orthogonality or broke down
                                (float64 then stays on for the rest of the call)       */
} rbo_info;

/* ---- sparse-sign sketch (Section 3 / 5.2; the paper's Count sketch with zeta
 *      nonzeros per column) ------------------------------------------------------
 * S is d x n; column r holds zeta distinct row indices with signs +-1, drawn
 * from the SplitMix64 stream (Steele, Lea & Flood 2014) seeded with `seed`:
 * row r owns outputs i = 64 r + c + 1 (c = 0..63) of that stream; output h gives
 * index ((h >> 32) * d) >> 32 and sign -1 iff bit 0 of h is set; repeated
 * indices are skipped.  The entries are hashed once per call (per GMRES solve)
 * into a per-tile transposed schedule in the call's workspace.  Values are +-1,
 * unscaled.                                                                        */
typedef struct rbo_sketch_s* rbo_sketch;

/* Create a sketch handle for matrices of up to n_max rows.  1 <= zeta <= d <= 4096.
 * The handle is library-owned (host memory only); destroy it with
 * rbo_sketch_destroy.  Errors: RBO_ERR_ARG.                                        */
int rbo_sketch_create(int64_t n_max, int32_t d, int32_t zeta, uint64_t seed, rbo_sketch* out);
/* Typed sketch (Section 5.2 compares these maps):
 *  RBO_SKETCH_SPARSE_SIGN: as rbo_sketch_create (d_inner ignored).
 *  RBO_SKETCH_GAUSSIAN: S (d x n) dense, S[k, r] = theta(seed, r, k, d) with theta =
 *    sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller, float32 arithmetic) from output
 *    i = r d + k + 1 of the SplitMix64 stream seeded with seed ^ 0x2545F4914F6CDD1D:
 *    u1 = fl32(h>>40 + 1/2) 2^-24, u2 = ((h >> 16) & 0xFFFFFF) 2^-24.  Entries are
 *    generated in the kernels, never stored.  1 <= d <= 256.
 *  RBO_SKETCH_COUNT_GAUSS: S = G C with C the d_inner x n Count sketch (the
 *    sparse-sign map with zeta = 1 and this seed) and G (d x d_inner) Gaussian with
 *    G[k, j] = theta(seed, j, k, d).  1 <= d <= 4096, 1 <= d_inner <= 4096.
 * zeta is used by SPARSE_SIGN only.  Errors: RBO_ERR_ARG, RBO_ERR_NOMEM.            */
int rbo_sketch_create_ex(int64_t n_max, int32_t d, int32_t type, int32_t zeta, int32_t d_inner,
                         uint64_t seed, rbo_sketch* out);
int rbo_sketch_destroy(rbo_sketch sk);

/* Materialise the entries of columns row0 .. row0+nrows-1 of S on the device, with
 * the same device code the sketch apply uses: idx (nrows x zeta, int32, row-major)
 * and sign (nrows x zeta, int8), both caller-owned device arrays.  For tests.
 * Count-Gauss: the entries of its Count stage (zeta = 1); Gaussian: RBO_ERR_ARG.
 * Errors: RBO_ERR_ARG, RBO_ERR_SKETCH, RBO_ERR_CUDA.                               */
int rbo_sketch_entries(rbo_sketch sk, int64_t row0, int64_t nrows, int32_t* idx, int8_t* sign,
                       void* stream);

/* out = S W  (d x k, column-major, ld d, caller-owned HOST array) for W (n x k,
 * device, ld ldw).  The step "v = Theta^T V" of RandHH (Section 5.2).
 * `precision` RBO_PREC_FP64 or RBO_PREC_MIXED (float32 accumulation).            */
int rbo_sketch_apply(rbo_sketch sk, int64_t n, int32_t k, const double* W, int64_t ldw,
                     double* out, int32_t precision, void* stream);

/* ---- tall-skinny Gram (the reduction of BCGS / CholQR, Figures 2a-2b) ----------
 * C = X^T Y (a x b, column-major ld a, caller-owned HOST array) for device
 * X (n x a, ld ldx) and Y (n x b, ld ldy); a, b <= 128.  Deterministic
 * (fixed-order cross-CTA tree).                                                   */
int rbo_gram(int64_t n, int32_t a, const double* X, int64_t ldx, int32_t b, const double* Y,
             int64_t ldy, double* C, void* stream);
/* The same Gram in a given precision: RBO_PREC_FP64 (as rbo_gram) or RBO_PREC_OZAKI (the
 * tensor-core digit products; a <= 64 and b <= 8, RBO_ERR_ARG otherwise).  A column
 * holding a non-finite value gives NaN in its row or column of C.                  */
int rbo_gram_ex(int64_t n, int32_t a, const double* X, int64_t ldx, int32_t b, const double* Y,
                int64_t ldy, double* C, int32_t precision, void* stream);

/* ---- tall-skinny Gram without allocation -------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that cannot
 * let a library allocate device memory -- applications whose HBM is owned by another
 * allocator (a framework pool that has reserved the free memory), loops that must not
 * pay the implicit synchronisation of cudaMalloc/cudaFree, programs with a memory
 * budget fixed at start-up.
 * C = X^T Y like rbo_gram, but C is a caller-owned DEVICE array (a x b, column-major,
 * ld a) and the call allocates nothing: its reduction scratch is one static 4 MiB
 * device array (RBO_NOALLOC_SCRATCH_BYTES) that every GPU loading the library keeps
 * until the process exits.  Limits: a <= 128, b <= 64, a * b <= 2048 (larger shapes
 * return RBO_ERR_ARG).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and caches it for that device; that first call
 * should come before any stream capture begins.  All calls share the array and it
 * keeps the last call's contents (each call re-zeroes the counters it needs), so
 * calls that overlap on the GPU -- different streams or host threads at the same
 * time -- race and must be serialised by the caller.  Every call ends with a
 * device-to-host copy of the status word and a synchronisation of `stream`.  The
 * cached address does not survive a cudaDeviceReset of that device.
 * Errors: RBO_ERR_ARG, RBO_ERR_NO_DEVICE, RBO_ERR_TIMEOUT, RBO_ERR_CUDA.            */
int rbo_gram_noalloc(int64_t n, int32_t a, const double* X, int64_t ldx, int32_t b,
                     const double* Y, int64_t ldy, double* C, void* stream);

/* ---- block orthogonalization ------------------------------------------------------
 * V (n x ncols, device, ld ldv) is overwritten by Q; R (ncols x ncols, column-major,
 * ld ldr >= ncols, caller-owned HOST array) receives the upper-triangular factor.
 * Blocks: if opts->v0, column 0 is normalised first; the remaining columns form
 * blocks of s columns (ncols - v0 must be a multiple of s; 1 <= s <= 64;
 * ncols <= 129).  n >= ncols is required.  `sk` may be shared between calls.
 * The sketch size times the panel width, d * s, must not exceed 12288 (the
 * per-warp sketch partials live in shared memory); the same bound applies to
 * rbo_sketch_apply (d * k) and rbo_sstep_gmres (d * s).
 *
 * one_stage (Section 5): per block, BCGS2 with RandCholQR (or CholQR2) as the
 *   first intra-block step and CholQR after the re-orthogonalization.
 * two_stage (Sections 6-7): big panels of s_hat columns (s | s_hat,
 *   s_hat | ncols - v0, s_hat <= 64) built from panels of s; each panel is projected
 *   against the finished big panels (BCGS) and preprocessed with RandBCGS2
 *   (sketched BCGS2 with Householder intra step, then forward substitution); each
 *   big panel is finished by CholQR, BCGS and CholQR.  s_hat == s is one-stage.
 * cholqr2: one-stage BCGS2 with CholQR2 as the first intra-block step; reports
 *   RBO_ERR_CHOL_BREAKDOWN with the failing block and column instead of
 *   producing NaNs (Section 5.1).
 * Errors: RBO_ERR_ARG, RBO_ERR_CHOL_BREAKDOWN, RBO_ERR_TIMEOUT, RBO_ERR_CUDA,
 *         RBO_ERR_NOMEM, RBO_ERR_SKETCH.                                           */
int rbo_block_orth_one_stage(rbo_sketch sk, int64_t n, int32_t ncols, int32_t s, double* V,
                             int64_t ldv, double* R, int64_t ldr, const rbo_opts* opts,
                             rbo_info* info, void* stream);
int rbo_block_orth_two_stage(rbo_sketch sk, int64_t n, int32_t ncols, int32_t s, int32_t s_hat,
                             double* V, int64_t ldv, double* R, int64_t ldr, const rbo_opts* opts,
                             rbo_info* info, void* stream);
int rbo_block_orth_cholqr2(int64_t n, int32_t ncols, int32_t s, double* V, int64_t ldv, double* R,
                           int64_t ldr, const rbo_opts* opts, rbo_info* info, void* stream);

/* ---- CSR matrix and matrix-powers kernel (Section 4) ----------------------------- */
typedef struct rbo_csr {
  int64_t n;              /* rows = columns                                          */
  int64_t nnz;            /* < 2^31                                                  */
  const int32_t* rowptr;  /* device, n+1 entries, rowptr[0] = 0                      */
  const int32_t* col;     /* device, nnz column indices in [0, n)                    */
  const double* val;      /* device, nnz values                                      */
} rbo_csr;

/* Monomial MPK: V[:, i] = (A D)^{i+1} v0 for i = 0..s-1, with D = diag(dscale) if
 * dscale != NULL (right Jacobi scaling: dscale = 1 / diag(A)) else D = I.
 * v0 (n), dscale (n) and V (n x s, ld ldv) are device arrays; v0 must not alias V.
 * Errors: RBO_ERR_ARG, RBO_ERR_CUDA.                                              */
int rbo_mpk_csr(const rbo_csr* A, const double* dscale, int32_t s, const double* v0, double* V,
                int64_t ldv, void* stream);

/* Shifts of the Newton matrix-powers basis (Section 4 names it as the stabler option
 * of Trilinos; Bai, Hu and Reichel 1994): the Ritz values (eigenvalues) of the k x k
 * upper Hessenberg H (host, column-major, ld >= k; entries below the subdiagonal are
 * ignored) in modified Leja order, as the real recurrence
 *   v_{i+1} = (A - alpha_i) v_i + beta_i v_{i-1},  i = 0..s-1,
 * alpha_i = Re theta_i, beta_i = (Im theta_i)^2 for the second value of a conjugate
 * pair and 0 otherwise (a pair cut by the s-th position keeps its real part).
 * alpha, beta: caller-owned host arrays of s doubles.  Host-only (no GPU needed).
 * Errors: RBO_ERR_ARG, RBO_ERR_NOT_CONVERGED (QR iteration did not converge).      */
int rbo_newton_shifts(const double* H, int64_t ld, int32_t k, int32_t s, double* alpha,
                      double* beta);

/* Recurrence of the Chebyshev matrix-powers basis (Sections 5 and 8 name it beside the
 * Newton basis; Joubert and Carey 1992), in the same form
 *   v_{i+1} = (A - alpha_i) v_i + beta_i v_{i-1},  i = 0..s-1:
 * v_k = p_k(A) v_0 with p_k(z) = 2 (e/2)^k T_k((z - c)/e) (T_k: Chebyshev polynomials of
 * the first kind), i.e. alpha_i = c, beta_0 = 0, beta_1 = -e^2/2, beta_i = -e^2/4.  The
 * ellipse (centre c on the real axis, half focal distance e; e^2 < 0 when the foci lie
 * on the line Re z = c) encloses the eigenvalues of the k x k upper Hessenberg H (host,
 * column-major, ld >= k): c is the midpoint of their real extent, the axes lie along
 * the real and imaginary directions, and among those ellipses it has the smallest
 * capacity (a + b)/2, a and b its semi-axes, e^2 = a^2 - b^2 (a real spectrum gives
 * the interval of the eigenvalues).
 * alpha, beta: caller-owned host arrays of s doubles.  Host-only (no GPU needed).
 * Errors: RBO_ERR_ARG, RBO_ERR_NOT_CONVERGED (QR iteration did not converge).      */
int rbo_chebyshev_shifts(const double* H, int64_t ld, int32_t k, int32_t s, double* alpha,
                         double* beta);

/* ---- s-step GMRES (Section 4, Figure 1) -------------------------------------------
 * (opts->preproc selects RandBCGS2 or BCGS-PIP for the two-stage panels)
 * Solves A x = b (b, x: device, n) with restart length m (s | m, m <= 128) and
 * right preconditioner opts->precond.  x holds x0 on entry (resume from a
 * previous solve) and the solution on exit.  s_hat == 0 or s_hat == s: one-stage
 * randomized BCGS2; s < s_hat (s | s_hat | m): two-stage with RandBCGS2.
 * opts->intra = RBO_INTRA_CHOLQR2 runs the one-stage scheme with CholQR2 instead of
 * RandCholQR (the deterministic baseline, which breaks down on ill-conditioned
 * monomial panels).  opts->basis selects the matrix-powers basis: monomial (the
 * paper's), or Newton / Chebyshev, whose first restart cycle runs standard GMRES to
 * obtain the Ritz values (rbo_newton_shifts, rbo_chebyshev_shifts) and whose later
 * panels use the shifted three-term recurrence (H = (Y + X B) X^-1).
 * The sketch has d = 4 (m + 1) rows, zeta = 8, seed 42 unless `sk` is given.
 * Converged when ||b - A x||_2 <= tol ||b||_2 (true residual).
 * Errors: RBO_ERR_ARG, RBO_ERR_NOT_CONVERGED, RBO_ERR_CHOL_BREAKDOWN, RBO_ERR_CUDA,
 *         RBO_ERR_NOMEM, RBO_ERR_TIMEOUT.                                          */
int rbo_sstep_gmres(const rbo_csr* A, const double* b, double* x, int32_t s, int32_t s_hat,
                    int32_t m, double tol, rbo_sketch sk, const rbo_opts* opts, rbo_info* info,
                    void* stream);

/* s-step GMRES with a caller-supplied right preconditioner M that has A's sparsity
 * pattern: Mval (device, A->nnz values in A's CSR order).  The matrix-powers kernel
 * applies A M (two SpMVs per basis vector; the operator stays linear, so s-step
 * GMRES stays valid, Section 4) and the solution update is x += M Q z.  Other
 * arguments, errors and convergence test as rbo_sstep_gmres; opts->precond is
 * ignored.  Used with the learned preconditioner below.                            */
int rbo_sstep_gmres_precond(const rbo_csr* A, const double* Mval, const double* b, double* x,
                            int32_t s, int32_t s_hat, int32_t m, double tol, rbo_sketch sk,
                            const rbo_opts* opts, rbo_info* info, void* stream);

/* ---- learned sparse-approximate-inverse preconditioner -----------------------------
 * Not in the paper: a graph network (3 message-passing layers, width 32, BF16
 * weights, FP32 activations and accumulation) maps the entries of A to the values
 * of a right preconditioner M on A's pattern, keeping the matrix-powers kernel
 * linear.  Nodes are rows of A, each stored entry (i, j) an edge from j to i; with
 * D = diag(A) and Ahat = D^-1 A the inputs are, per node, the off-diagonal row and
 * column sums of |Ahat| and, per edge, (Ahat_ij, Ahat_ji, [i == j]); the output is
 * M_ij = (network output + [i == j]) / A_ii, so an untrained network (zero output
 * layer) is the Jacobi preconditioner.  Training minimises
 * mean_k ||r_k - A M r_k||^2 / ||r_k||^2 over residual vectors r_k (Adam, FP32 master
 * weights).  A must be square with a nonzero diagonal and a structurally symmetric
 * pattern (RBO_ERR_ARG otherwise).  The handle owns ~0.3 MB of device memory;
 * calls use the per-device workspace arena.  Parameters are a flat float vector of
 * rbo_gnn_param_count() values in the order Wn(32x2) bn We(32x3) be, then per layer
 * Wm(32x64) bm Wh(32x64) bh, then wo(96) bo (row-major matrices).  The message and
 * node layers and their backward run on the tensor cores: each FP32 activation is
 * split into three BF16 pieces, whose products with the BF16 weights are exact, and
 * the sums are FP32, so the results agree with an FP32 evaluation.              */
typedef struct rbo_gnn_s* rbo_gnn;
int rbo_gnn_param_count(void);
/* Random He-scaled hidden weights from `seed`, zero biases and output layer.       */
int rbo_gnn_create(uint64_t seed, rbo_gnn* out);
int rbo_gnn_destroy(rbo_gnn g);
/* FP32 master weights from / to host memory (set also resets the Adam state).      */
int rbo_gnn_set_params(rbo_gnn g, const float* host);
int rbo_gnn_get_params(rbo_gnn g, float* host);
/* Mval (device, A->nnz) = M on A's pattern for the current weights.                */
int rbo_gnn_infer(rbo_gnn g, const rbo_csr* A, double* Mval, void* stream);
/* Loss over the nr residual columns of R (device, n x nr, ld ldr >= n, nr <= 64)
 * and its gradient with respect to the parameters (grad_host may be NULL).          */
int rbo_gnn_loss_grad(rbo_gnn g, const rbo_csr* A, const double* R, int32_t nr, int64_t ldr,
                      double* loss, float* grad_host, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on that loss;
 * *loss receives the loss before the step.                                        */
int rbo_gnn_train_step(rbo_gnn g, const rbo_csr* A, const double* R, int32_t nr, int64_t ldr,
                       float lr, double* loss, void* stream);

/* ---- per-kernel timing ---------------------------------------------------------------
 * When enabled, every kernel the library enqueues is bracketed by two CUDA events on
 * its stream and tagged with its algorithmic DRAM bytes (each n-row column read or
 * written once) and floating-point operations.  Totals accumulate per kernel kind
 * until rbo_profile_reset.  Reading drains pending events (synchronising on them).
 * Process-wide; not for concurrent calls from several host threads.              */
#define RBO_PROF_ROWPASS 0  /* the fused tall-skinny row pass (Gram / update / TRSM / sketch) */
#define RBO_PROF_SPMV    1  /* CSR SpMV of the matrix-powers kernel and residuals           */
#define RBO_PROF_VECTOR  2  /* small vector kernels (Jacobi setup, x update, scaling)       */
#define RBO_PROF_OZAKI   3  /* the tensor-core Gram passes of RBO_PREC_OZAKI (also counted
                               by role below)                                           */
/* Row passes are also accumulated by role under kind RBO_PROF_PASS + role:
 * 1..6 one-stage P1 (Gram C1), P2 (update + sketch), P3 (TRSM R_hat + Gram),
 * P4 (TRSM R' + Gram C2), P5 (re-orthogonalization update + Gram), P6 (final TRSM);
 * 7..12 two-stage T1..T6 (same roles per big panel); 13 normalisations; 0 other.   */
#define RBO_PROF_PASS    8
int rbo_profile_enable(int on);
int rbo_profile_reset(void);
int rbo_profile_read(int32_t kind, int64_t* launches, double* ms, double* bytes, double* flops);

/* ---- housekeeping ------------------------------------------------------------------ */
const char* rbo_status_string(int status);
/* Free the calling thread's current device's workspace arena. */
int rbo_release_workspace(void);
/* Library version string and the sm architecture it was compiled for. */
const char* rbo_version(void);
/* Name and description of the last CUDA error a call of this host thread met
 * (empty if none); valid until the next failing call. */
const char* rbo_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RBO_H */

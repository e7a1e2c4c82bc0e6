// Host orchestration of the block orthogonalization schemes as sequences of row
// passes (see rowpass.cu).  All work is enqueued on one stream; small factors stay
// in device buffers and are consumed by later passes, so there is no host round
// trip inside a block.
//
// One-stage BCGS2 with RandCholQR (Sections 4-5), block j with p previous columns:
//   P1  C1 = Q^T W                                     (BCGS Gram)
//   P2  W = W - Q C1 ; w = S W ; R_hat = HH(w)          (BCGS update + sketch, RandHH)
//   P3  W = W R_hat^{-1} ; G = W^T W ; R' = chol(G)     (RandHH TRSM + CholQR Gram)
//   P4  W = W R'^{-1} ; C2 = Q^T W                      (CholQR TRSM + re-orth Gram)
//   P5  W = W - Q C2 ; G2 = W^T W ; R2 = chol(G2)       (re-orth update + CholQR Gram)
//       R[:p, j] = C1 + C2 R' R_hat ; R_jj = R2 R' R_hat
//   P6  W = W R2^{-1}                                    (final TRSM)
// CholQR2 as the first intra step replaces the sketch of P2 by G = W^T W and
// R_hat = chol(G).
#include <algorithm>

#include "rbo_internal.cuh"

namespace rbo {

// The sparse part of a sketch that the row pass scatters (sparse-sign, or the Count
// stage of Count-Gauss): rows and nonzeros per column; 0 rows for none.
static void sched_shape(int type, int d, int d_inner, int zeta, int* ds, int* zs) {
  *ds = type == RBO_SKETCH_SPARSE_SIGN ? d : (type == RBO_SKETCH_COUNT_GAUSS ? d_inner : 0);
  *zs = type == RBO_SKETCH_SPARSE_SIGN ? zeta : 1;
}

size_t orth_ctx_bytes(int pmax, int kmax, int d, int64_t n, int zeta, int type, int d_inner) {
  size_t pk = (size_t)std::max(pmax, 1) * kmax, kk = (size_t)kmax * kmax;
  size_t dd = (size_t)std::max(d, 1) * kmax;
  int ds = 0, zs = 0;
  sched_shape(type, d, d_inner, zeta, &ds, &zs);
  const size_t tab =
      (d > 0 && ds > 0) ? sketch_sched_bytes(n, rowpass_sketch_T(pmax, kmax, ds, zs), ds, zs) + 256 : 0;
  return (2 * pk + 6 * kk + dd + pk + kk) * 8 + 16 * 256 + tab;
}

void set_sketch(RowPass& r, const OrthCtx& c) {
  r.sk_seed = c.seed;
  if (c.sk_type == RBO_SKETCH_GAUSSIAN) {
    r.sk_gd = c.d;
  } else if (c.sk_type == RBO_SKETCH_COUNT_GAUSS) {
    r.sk_d = c.d_inner; r.sk_zeta = 1; r.sk = c.sk; r.sk_cg = c.d;
  } else {
    r.sk_d = c.d; r.sk_zeta = c.zeta; r.sk = c.sk;
  }
}

int orth_max_L(int pmax, int kmax, int d) {
  // Z of at most (pmax + kmax) x kmax plus a d x kmax sketch (d: the largest of the
  // final and the scattered sketch rows)
  return (pmax + kmax) * kmax + std::max(d, 0) * kmax;
}

int orth_ctx_alloc(OrthCtx& c, int pmax, int kmax, int64_t n) {
  c.pmax = pmax;
  c.kmax = kmax;
  size_t pk = (size_t)std::max(pmax, 1) * kmax, kk = (size_t)kmax * kmax;
  size_t dd = (size_t)std::max(c.d, 1) * kmax;
  c.C1 = (double*)c.ar->take(pk * 8);
  c.C2 = (double*)c.ar->take(pk * 8);
  c.Rh = (double*)c.ar->take(kk * 8);
  c.Rp = (double*)c.ar->take(kk * 8);
  c.R2 = (double*)c.ar->take(kk * 8);
  c.T = (double*)c.ar->take(kk * 8);
  c.GB = (double*)c.ar->take(kk * 8);
  c.qs = (double*)c.ar->take(dd * 8);
  c.tmp = (double*)c.ar->take((pk + kk) * 8);
  if (!c.C1 || !c.C2 || !c.Rh || !c.Rp || !c.R2 || !c.T || !c.GB || !c.qs || !c.tmp)
    return RBO_ERR_NOMEM;
  c.sk = SketchSched();
  int ds = 0, zs = 0;
  sched_shape(c.sk_type, c.d, c.d_inner, c.zeta, &ds, &zs);
  if (c.d > 0 && ds > 0) {
    // the sparse sketch is a fixed operator for the call: hashed and transposed once
    const int T = rowpass_sketch_T(pmax, kmax, ds, zs);
    uint8_t* rec = (uint8_t*)c.ar->take(sketch_sched_bytes(n, T, ds, zs));
    if (!rec) return RBO_ERR_NOMEM;
    const int e = sketch_sched_launch(n, T, ds, zs, c.seed, rec, c.ar->status, c.st);
    if (e != RBO_OK) return e;
    c.launches += 1;
    c.sk.rec = rec;
    c.sk.T = T;
    c.sk.mcap = sketch_sched_mcap(T, ds, zs);
    c.sk.rec_bytes = sketch_sched_rec_bytes(T, ds, zs);
  }
  return RBO_OK;
}

#define RBO_TRY(x)             \
  do {                         \
    int _e = (x);              \
    if (_e != RBO_OK) return _e; \
  } while (0)

int normalise_column(OrthCtx& c, int64_t n, double* v, double* Rdev, int ldR, int col0) {
  const int64_t ldeven = (n + 1) & ~int64_t(1);  // only column 0 is used
  RowPass g;
  g.df64 = c.df64;
  g.ozaki = c.ozaki;
  g.tag = 13;
  g.n = n;
  g.Y = v;
  g.ldy = ldeven;
  g.b = 1;
  g.acc_y = 1;
  g.epi.op = EPI_CHOL;
  g.epi.out_r = c.R2;
  g.epi.stage = RBO_STAGE_V0;
  g.epi.block = -1;
  g.epi.asm_op = ASM_DIAG;
  g.epi.Rfull = Rdev;
  g.epi.ldR = ldR;
  g.epi.p = col0;
  g.epi.col0 = col0;
  RBO_TRY(rowpass_launch(g, c.ar, c.st, &c.launches));
  RowPass s;
  s.df64 = c.df64;
  s.ozaki = c.ozaki;
  s.tag = 13;
  s.n = n;
  s.Y = v;
  s.ldy = ldeven;
  s.b = 1;
  s.Tri = c.R2;
  s.write_y = 1;
  return rowpass_launch(s, c.ar, c.st, &c.launches);
}

int one_stage_block(OrthCtx& c, int64_t n, const double* Q, int64_t ldq, int p, double* W,
                    int64_t ldw, int k, int intra, double* Rdev, int ldR, int col0, int blk) {
  if (p > c.pmax || k > c.kmax) return RBO_ERR_ARG;
  const bool rand = intra == RBO_INTRA_RANDCHOLQR;
  // P1: C1 = Q^T W
  if (p > 0) {
    RowPass r;
    r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 1;
    r.n = n; r.X = Q; r.ldx = ldq; r.a = p; r.Y = W; r.ldy = ldw; r.b = k;
    r.acc_x = 1;
    r.mixed = c.mixed;
    r.epi.op = EPI_STORE; r.epi.out = c.C1; r.epi.out_ld = p;
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  }
  // P2: W = W - Q C1, then sketch -> R_hat (or Gram -> chol for CholQR2)
  {
    RowPass r;
    r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 2;
    r.n = n; r.X = Q; r.ldx = ldq; r.a = p; r.Y = W; r.ldy = ldw; r.b = k;
    if (p > 0) { r.C = c.C1; r.write_y = 1; }
    if (rand) {
      set_sketch(r, c);
      r.mixed = c.mixed;
      r.epi.op = EPI_HH; r.epi.out_r = c.Rh; r.epi.stage = RBO_STAGE_INTRA; r.epi.block = blk;
    } else {
      r.acc_y = 1;
      r.epi.op = EPI_CHOL; r.epi.out_r = c.Rh; r.epi.stage = RBO_STAGE_INTRA; r.epi.block = blk;
    }
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  }
  // P3: W = W R_hat^{-1}; R' = chol(W^T W)
  {
    RowPass r;
    r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 3;
    r.n = n; r.Y = W; r.ldy = ldw; r.b = k;
    r.Tri = c.Rh; r.write_y = 1; r.acc_y = 1;
    r.epi.op = EPI_CHOL; r.epi.out_r = c.Rp; r.epi.block = blk;
    r.epi.stage = rand ? RBO_STAGE_INTRA : RBO_STAGE_INTRA2;
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  }
  Epilogue fin;
  fin.op = EPI_CHOL; fin.out_r = c.R2; fin.stage = RBO_STAGE_FINAL; fin.block = blk;
  fin.asm_op = ASM_ONE_STAGE;
  fin.C1 = c.C1; fin.ldc1 = std::max(p, 1);
  fin.C2 = c.C2; fin.ldc2 = std::max(p, 1);
  fin.Rh = c.Rh; fin.Rp = c.Rp;
  fin.Rfull = Rdev; fin.ldR = ldR; fin.p = p; fin.col0 = col0;
  if (p > 0) {
    // P4: W = W R'^{-1}; C2 = Q^T W
    {
      RowPass r;
      r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 4;
      r.n = n; r.X = Q; r.ldx = ldq; r.a = p; r.Y = W; r.ldy = ldw; r.b = k;
      r.Tri = c.Rp; r.write_y = 1; r.acc_x = 1;
      r.epi.op = EPI_STORE; r.epi.out = c.C2; r.epi.out_ld = p;
      RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
    }
    // P5: W = W - Q C2; R2 = chol(W^T W); assemble R
    {
      RowPass r;
      r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 5;
      r.n = n; r.X = Q; r.ldx = ldq; r.a = p; r.Y = W; r.ldy = ldw; r.b = k;
      r.C = c.C2; r.write_y = 1; r.acc_y = 1; r.small_coeffs = 1;
      r.epi = fin;
      RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
    }
  } else {
    // no previous basis: W = W R'^{-1} and its Gram in one pass
    RowPass r;
    r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 4;
    r.n = n; r.Y = W; r.ldy = ldw; r.b = k;
    r.Tri = c.Rp; r.write_y = 1; r.acc_y = 1;
    r.epi = fin;
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  }
  // P6: Q_j = W R2^{-1}
  RowPass r;
  r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 6;
  r.n = n; r.Y = W; r.ldy = ldw; r.b = k;
  r.Tri = c.R2; r.write_y = 1;
  return rowpass_launch(r, c.ar, c.st, &c.launches);
}

// ---- two-stage (Sections 6-7) -----------------------------------------------------------
// Per panel j of a big panel with P finished columns Q:
//   T1  C1_j = Q^T V_j
//   T2  Vh_j = V_j - Q C1_j ; v_j = S Vh_j ; sketched BCGS2-HH -> T(:, j), q_j
//   T3  Qbar_j = (Vh_j - Qbar_{<j} T_{<j,j}) T_jj^{-1} ; block column of G_B = Qbar^T Qbar
// At the end of the big panel (R' = chol(G_B) from the last T3):
//   T4  Qh = Qbar R'^{-1} ; C2 = Q^T Qh
//   T5  W = Qh - Q C2 ; R2 = chol(W^T W) ; R_QB = C1 + C2 R' T, R_BB = R2 R' T
//   T6  Q_B = W R2^{-1}
int bigpanel_add(OrthCtx& c, BigPanel& bp, int k) {
  const int K = bp.K, cols = bp.cols, P = bp.P;
  if (cols + k > K || P > c.pmax || K > c.kmax) return RBO_ERR_ARG;
  double* W = bp.VB + (int64_t)cols * bp.ldv;
  if (P > 0) {
    RowPass r;
    r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 7;
    r.n = bp.n; r.X = bp.Q; r.ldx = bp.ldq; r.a = P; r.Y = W; r.ldy = bp.ldv; r.b = k;
    r.acc_x = 1;
    r.mixed = c.mixed;
    r.epi.op = EPI_STORE; r.epi.out = c.C1; r.epi.out_ld = P; r.epi.col_off = cols;
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  }
  if (c.pip) {
    // BCGS-PIP preprocessing (Section 7.1): Vh = V - Q C1, then one reduction of
    // [Qbar_{<j}, Vh]^T Vh whose epilogue factors the Pythagorean Gram G - P^T P.
    // The reduction stays float64 in every precision mode: its Cholesky loses
    // kappa^2 of the accumulation precision.
    if (P > 0) {
      RowPass r;
      r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 8;
      r.n = bp.n; r.X = bp.Q; r.ldx = bp.ldq; r.a = P; r.Y = W; r.ldy = bp.ldv; r.b = k;
      r.C = c.C1 + (size_t)cols * P; r.ldc = P; r.write_y = 1;
      RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
    }
    RowPass r;
    r.tag = 14;
    r.n = bp.n; r.X = bp.VB; r.ldx = bp.ldv; r.a = cols; r.Y = W; r.ldy = bp.ldv; r.b = k;
    r.acc_x = cols > 0 ? 1 : 0; r.acc_y = 1;
    r.epi.op = EPI_PIP; r.epi.T = c.T; r.epi.K = K; r.epi.poff = cols;
    r.epi.stage = RBO_STAGE_PREPROC; r.epi.block = bp.blk;
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  } else {
    RowPass r;
    r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 8;
    r.n = bp.n; r.X = bp.Q; r.ldx = bp.ldq; r.a = P; r.Y = W; r.ldy = bp.ldv; r.b = k;
    if (P > 0) { r.C = c.C1 + (size_t)cols * P; r.ldc = P; r.write_y = 1; }
    set_sketch(r, c);
    r.mixed = c.mixed;
    r.epi.op = EPI_SKB2; r.epi.qs = c.qs; r.epi.T = c.T; r.epi.K = K; r.epi.poff = cols;
    r.epi.stage = RBO_STAGE_BIGPANEL; r.epi.block = bp.blk;
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  }
  {
    RowPass r;
    r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 9;
    r.n = bp.n; r.X = bp.VB; r.ldx = bp.ldv; r.a = cols; r.Y = W; r.ldy = bp.ldv; r.b = k;
    if (cols > 0) { r.C = c.T + (size_t)cols * K; r.ldc = K; r.acc_x = 1; }
    r.Tri = c.T + cols + (size_t)cols * K; r.ldtri = K;
    r.write_y = 1; r.acc_y = 1;
    r.epi.op = EPI_GB; r.epi.GB = c.GB; r.epi.K = K; r.epi.poff = cols;
    r.epi.last = (cols + k == K) ? 1 : 0;
    r.epi.out_rp = c.Rp; r.epi.block = bp.blk;
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  }
  bp.cols += k;
  return RBO_OK;
}

int bigpanel_finish(OrthCtx& c, BigPanel& bp, double* Rdev, int ldR, int col0, double* coords,
                    int ldcoords) {
  const int K = bp.K, P = bp.P;
  if (bp.cols != K) return RBO_ERR_ARG;
  Epilogue fin;
  fin.op = EPI_CHOL; fin.out_r = c.R2; fin.stage = RBO_STAGE_FINAL; fin.block = bp.blk;
  fin.asm_op = ASM_TWO_STAGE;
  fin.C1 = c.C1; fin.ldc1 = std::max(P, 1);
  fin.C2 = c.C2; fin.ldc2 = std::max(P, 1);
  fin.Rh = c.T; fin.Rp = c.Rp;
  fin.Rfull = Rdev; fin.ldR = ldR; fin.p = P; fin.col0 = col0;
  fin.coords = coords; fin.ldcoords = ldcoords;
  if (P > 0) {
    {
      RowPass r;
      r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 10;
      r.n = bp.n; r.X = bp.Q; r.ldx = bp.ldq; r.a = P; r.Y = bp.VB; r.ldy = bp.ldv; r.b = K;
      r.Tri = c.Rp; r.write_y = 1; r.acc_x = 1;
      r.epi.op = EPI_STORE; r.epi.out = c.C2; r.epi.out_ld = P;
      RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
    }
    {
      RowPass r;
      r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 11;
      r.n = bp.n; r.X = bp.Q; r.ldx = bp.ldq; r.a = P; r.Y = bp.VB; r.ldy = bp.ldv; r.b = K;
      r.C = c.C2; r.write_y = 1; r.acc_y = 1; r.small_coeffs = 1;
      r.epi = fin;
      RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
    }
  } else {
    RowPass r;
    r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 10;
    r.n = bp.n; r.Y = bp.VB; r.ldy = bp.ldv; r.b = K;
    r.Tri = c.Rp; r.write_y = 1; r.acc_y = 1;
    r.epi = fin;
    RBO_TRY(rowpass_launch(r, c.ar, c.st, &c.launches));
  }
  RowPass r;
  r.df64 = c.df64; r.ozaki = c.ozaki; r.tag = 12;
  r.n = bp.n; r.Y = bp.VB; r.ldy = bp.ldv; r.b = K;
  r.Tri = c.R2; r.write_y = 1;
  return rowpass_launch(r, c.ar, c.st, &c.launches);
}

}  // namespace rbo

// Block orthogonalization schemes, written step by step (oracle; test infrastructure).
// Each function restates the passage it follows; V = QR with Q^T Q = I and R upper
// triangular with a non-negative diagonal (Figure 1 caption); v0 means column 0 is the
// single starting vector V_0 = [v_0] (Table 1), normalised (CholQR of one column)
// before the blocks of s columns.
#include "orth.hpp"

namespace oracle {

// Figure 2a, BCGS: C = Q^T W; W_hat = W - Q C (the two operations Section 9 lists).
void bcgs(const Mat& Q, const Mat& W, Mat& C, Mat& What) {
  if (Q.n == 0) {
    C = Mat(0, W.n);
    What = W;
    return;
  }
  C = matmul_tn(Q, W);
  What = sub(W, matmul(Q, C));
}

// Figure 2b, CholQR: G = W^T W; R = chol(G) (upper, G = R^T R); Q = W R^{-1} (Sec. 5.1).
void cholqr(const Mat& W, Mat& Q, Mat& R, const char* where) {
  const Mat G = matmul_tn(W, W);
  const int info = cholesky_upper(G, R);
  if (info >= 0) throw Breakdown{info, where};
  Q = solve_right_upper(W, R);
}

// CholQR twice: [Q1, R1] = CholQR(W); [Q, R2] = CholQR(Q1); R = R2 R1 (Section 5.1).
void cholqr2(const Mat& W, Mat& Q, Mat& R) {
  Mat Q1, R1, R2;
  cholqr(W, Q1, R1, "cholqr2-first");
  cholqr(Q1, Q, R2, "cholqr2-second");
  R = matmul(R2, R1);
}

// Figure 4a, RandHH: w = S W; R_hat = R of Householder QR(w); Q_bar = W R_hat^{-1}.
void rand_hh(const Mat& W, const Sketch& S, Mat& Qbar, Mat& Rh) {
  const Mat w = S.apply(W);
  householder_qr(w, Rh, nullptr);
  Qbar = solve_right_upper(W, Rh);
}

// Figure 4b, RandCholQR: RandHH, then CholQR of Q_bar; R = R' R_hat (Prop. 5.2).
void rand_cholqr(const Mat& W, const Sketch& S, Mat& Q, Mat& R) {
  Mat Qbar, Rh, Rp;
  rand_hh(W, S, Qbar, Rh);
  cholqr(Qbar, Q, Rp, "randcholqr");
  R = matmul(Rp, Rh);
}

// Figure 2c, one block of BCGS2 (Section 4, the BCGSI+ structure):
//   [C1, W] = BCGS(Q, V_j); [Qh, Rh] = IntraBlk(W); [C2, Wt] = BCGS(Q, Qh);
//   [Q_j, R2] = CholQR(Wt); R_{Q,j} = C1 + C2 Rh, R_jj = R2 Rh.
void bcgs2_block(const Mat& Q, const Mat& Vj, int intra, const Sketch* S, Mat& Qj, Mat& Rtop, Mat& Rjj) {
  Mat C1, W, Qh, Rh, C2, Wt, R2;
  bcgs(Q, Vj, C1, W);
  if (intra == 0) rand_cholqr(W, *S, Qh, Rh);
  else cholqr2(W, Qh, Rh);
  bcgs(Q, Qh, C2, Wt);
  cholqr(Wt, Qj, R2, "final-cholqr");
  Rtop = add(C1, matmul(C2, Rh));
  Rjj = matmul(R2, Rh);
}

static void place(Mat& Q, Mat& R, const Mat& Qj, const Mat& Rtop, const Mat& Rjj, int64_t p) {
  for (int64_t j = 0; j < Qj.n; ++j)
    for (int64_t i = 0; i < Q.m; ++i) Q(i, p + j) = Qj(i, j);
  for (int64_t j = 0; j < Rjj.n; ++j) {
    for (int64_t i = 0; i < p; ++i) R(i, p + j) = Rtop(i, j);
    for (int64_t i = 0; i < Rjj.m; ++i) R(p + i, p + j) = Rjj(i, j);
  }
}

static int64_t start(const Mat& V, bool v0, Mat& Q, Mat& R) {
  Q = Mat(V.m, V.n);
  R = Mat(V.n, V.n);
  if (!v0) return 0;
  Mat q, r;
  cholqr(cols(V, 0, 1), q, r, "v0");
  for (int64_t i = 0; i < V.m; ++i) Q(i, 0) = q(i, 0);
  R(0, 0) = r(0, 0);
  return 1;
}

// One-stage BCGS2 over blocks of s columns (Section 5); intra 0: RandCholQR first
// intra-block step (Figure 4b), 1: CholQR2 (the deterministic baseline).  A Cholesky
// breakdown stops the scheme and is reported with its block and column.
OrthResult block_orth_one_stage(const Mat& V, int s, const Sketch* S, int intra, bool v0) {
  OrthResult out;
  int64_t p = 0;
  try {
    p = start(V, v0, out.Q, out.R);
  } catch (const Breakdown& e) {
    out.ok = false;
    out.breakdown_column = e.column;
    out.where = e.where;
    return out;
  }
  if ((V.n - p) % s != 0) throw std::runtime_error("columns after v0 must be a multiple of s");
  int blk = 0;
  while (p < V.n) {
    Mat Qj, Rtop, Rjj;
    try {
      bcgs2_block(cols(out.Q, 0, p), cols(V, p, s), intra, S, Qj, Rtop, Rjj);
    } catch (const Breakdown& e) {
      out.ok = false;
      out.breakdown_block = blk;
      out.breakdown_column = e.column;
      out.where = e.where;
      return out;
    }
    place(out.Q, out.R, Qj, Rtop, Rjj, p);
    p += s;
    ++blk;
  }
  return out;
}

// Section 7.2, BCGS2 with a Householder intra-block step on sketched vectors: qs (d x p')
// the sketched orthonormal basis of the big panel's earlier panels, v (d x k) the sketch
// of the new panel; v = qs T_col + q_new T_jj with [qs, q_new] orthonormal.
static void sketched_bcgs2_hh(const Mat& qs, const Mat& v, Mat& qn, Mat& Tcol, Mat& Tjj) {
  if (qs.n == 0) {
    householder_qr(v, Tjj, &qn);
    Tcol = Mat(0, v.n);
    return;
  }
  const Mat c1 = matmul_tn(qs, v);
  const Mat v1 = sub(v, matmul(qs, c1));
  const Mat c2 = matmul_tn(qs, v1);
  const Mat v2 = sub(v1, matmul(qs, c2));
  householder_qr(v2, Tjj, &qn);
  Tcol = add(c1, c2);
}

// Section 7.1, BCGS with the Pythagorean inner product: one reduction gives
// P = Qbar^T Vh and G = Vh^T Vh; the Gram of the projected block is G - P^T P, whose
// Cholesky factor is T_jj; Qbar_j = (Vh - Qbar P) T_jj^{-1} (CholQR without an earlier
// panel, the section's footnote).
static void bcgs_pip(const Mat& Qbar, const Mat& Vh, Mat& Qbj, Mat& P, Mat& Tjj) {
  P = Qbar.n > 0 ? matmul_tn(Qbar, Vh) : Mat(0, Vh.n);
  const Mat G = matmul_tn(Vh, Vh);
  const Mat Gp = Qbar.n > 0 ? sub(G, matmul_tn(P, P)) : G;
  const int info = cholesky_upper(Gp, Tjj);
  if (info >= 0) throw Breakdown{info, "bcgs-pip"};
  Qbj = solve_right_upper(Qbar.n > 0 ? sub(Vh, matmul(Qbar, P)) : Vh, Tjj);
}

static Mat hcat(const Mat& A, const Mat& B) {
  Mat C(A.n > 0 ? A.m : B.m, A.n + B.n);
  for (int64_t j = 0; j < A.n; ++j)
    for (int64_t i = 0; i < C.m; ++i) C(i, j) = A(i, j);
  for (int64_t j = 0; j < B.n; ++j)
    for (int64_t i = 0; i < C.m; ++i) C(i, A.n + j) = B(i, j);
  return C;
}

TwoStageBigPanel::TwoStageBigPanel(const Mat& Q_, const Sketch* S_, int K_, int pip_)
    : Q(&Q_), S(S_), K(K_), pip(pip_), Qbar(Q_.m, 0), qs(S_ ? S_->d : 0, 0), T(K_, K_), C1(Q_.n, K_) {}

// Per panel j: [C1_j, Vh_j] = BCGS(Q, V_j) (inter big-panel BCGS), then the
// preprocessing: RandBCGS2 (Section 7.2: v_j = S Vh_j; [q_j, T_{<j,j}, T_jj] =
// sketched BCGS2-HH(qs, v_j); Qbar_j = (Vh_j - Qbar_{<j} T_{<j,j}) T_jj^{-1}, the
// forward substitution Qbar = Vh T^{-1} of the Appendix) or BCGS-PIP (Section 7.1).
Mat TwoStageBigPanel::add_panel(const Mat& Vj) {
  const int64_t k = Vj.n, a = cols;
  Mat C1j, Vh;
  bcgs(*Q, Vj, C1j, Vh);
  for (int64_t j = 0; j < k; ++j)
    for (int64_t i = 0; i < C1j.m; ++i) C1(i, a + j) = C1j(i, j);
  Mat Qbj, Tcol, Tjj;
  if (pip) {
    bcgs_pip(Qbar, Vh, Qbj, Tcol, Tjj);
  } else {
    Mat qn;
    sketched_bcgs2_hh(qs, S->apply(Vh), qn, Tcol, Tjj);
    Qbj = solve_right_upper(Qbar.n > 0 ? sub(Vh, matmul(Qbar, Tcol)) : Vh, Tjj);
    qs = hcat(qs, qn);
  }
  for (int64_t j = 0; j < k; ++j) {
    for (int64_t i = 0; i < a; ++i) T(i, a + j) = Tcol(i, j);
    for (int64_t i = 0; i < k; ++i) T(a + i, a + j) = Tjj(i, j);
  }
  Qbar = hcat(Qbar, Qbj);
  cols += (int)k;
  return Qbj;
}

// End of the big panel: [Qh_B, R'] = CholQR(Qbar_B); [C2, Wt] = BCGS(Q, Qh_B);
// [Q_B, R2] = CholQR(Wt); R_{Q,B} = C1 + C2 R' T, R_BB = R2 R' T; the coordinates of
// Qbar_B in [Q, Q_B] are [C2 R'; R2 R'].
void TwoStageBigPanel::finish(Mat& QB, Mat& RQB, Mat& RBB, Mat& coords) {
  const int64_t Kc = cols;
  Mat Tk(Kc, Kc);
  for (int64_t j = 0; j < Kc; ++j)
    for (int64_t i = 0; i < Kc; ++i) Tk(i, j) = T(i, j);
  Mat Qh, Rp, C2, Wt, R2;
  cholqr(Qbar, Qh, Rp, "bigpanel-cholqr");
  bcgs(*Q, Qh, C2, Wt);
  cholqr(Wt, QB, R2, "bigpanel-final-cholqr");
  const Mat RpT = matmul(Rp, Tk);
  RQB = add(oracle::cols(C1, 0, Kc), matmul(C2, RpT));
  RBB = matmul(R2, RpT);
  const Mat top = matmul(C2, Rp), bot = matmul(R2, Rp);
  coords = Mat(top.m + bot.m, Kc);
  for (int64_t j = 0; j < Kc; ++j) {
    for (int64_t i = 0; i < top.m; ++i) coords(i, j) = top(i, j);
    for (int64_t i = 0; i < bot.m; ++i) coords(top.m + i, j) = bot(i, j);
  }
}

// Two-stage block orthogonalization (Figure 6, Section 6): big panels of s_hat columns
// made of panels of s, preprocessed by RandBCGS2 (pip = 0) or BCGS-PIP (pip = 1).
OrthResult block_orth_two_stage(const Mat& V, int s, int s_hat, const Sketch* S, bool v0, int pip) {
  OrthResult out;
  int64_t p = 0;
  try {
    p = start(V, v0, out.Q, out.R);
  } catch (const Breakdown& e) {
    out.ok = false;
    out.breakdown_column = e.column;
    out.where = e.where;
    return out;
  }
  if ((V.n - p) % s_hat != 0 || s_hat % s != 0)
    throw std::runtime_error("columns after v0 must be a multiple of s_hat, and s_hat of s");
  int big = 0;
  while (p < V.n) {
    const Mat Qp = cols(out.Q, 0, p);
    TwoStageBigPanel bp(Qp, S, s_hat, pip);
    Mat QB, RQB, RBB, coords;
    try {
      for (int j = 0; j < s_hat / s; ++j) bp.add_panel(cols(V, p + j * s, s));
      bp.finish(QB, RQB, RBB, coords);
    } catch (const Breakdown& e) {
      out.ok = false;
      out.breakdown_block = big;
      out.breakdown_column = e.column;
      out.where = e.where;
      return out;
    }
    place(out.Q, out.R, QB, RQB, RBB, p);
    p += s_hat;
    ++big;
  }
  return out;
}

}  // namespace oracle

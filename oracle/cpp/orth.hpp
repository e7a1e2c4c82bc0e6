// Block orthogonalization schemes of the oracle (test infrastructure); see orth.cpp.
#pragma once

#include "common.hpp"

namespace oracle {

struct OrthResult {
  Mat Q, R;
  bool ok = true;
  int breakdown_block = -1, breakdown_column = -1;
  const char* where = "";
};

// BCGS (Figure 2a): C = Q^T W, W_hat = W - Q C.
void bcgs(const Mat& Q, const Mat& W, Mat& C, Mat& What);
// CholQR (Figure 2b): G = W^T W, R = chol(G), Q = W R^{-1}; throws Breakdown.
void cholqr(const Mat& W, Mat& Q, Mat& R, const char* where);
void cholqr2(const Mat& W, Mat& Q, Mat& R);
// RandHH (Figure 4a) and RandCholQR (Figure 4b).
void rand_hh(const Mat& W, const Sketch& S, Mat& Qbar, Mat& Rh);
void rand_cholqr(const Mat& W, const Sketch& S, Mat& Q, Mat& R);
// One block of BCGS2 with a first intra-block step: intra = 0 RandCholQR, 1 CholQR2.
void bcgs2_block(const Mat& Q, const Mat& Vj, int intra, const Sketch* S, Mat& Qj, Mat& Rtop, Mat& Rjj);

OrthResult block_orth_one_stage(const Mat& V, int s, const Sketch* S, int intra, bool v0);

// One big panel of the two-stage scheme (Sections 6-7).
struct TwoStageBigPanel {
  const Mat* Q;          // the earlier final basis (n x p)
  const Sketch* S;       // null for BCGS-PIP
  int K, pip;            // big-panel width, preprocessing (0 RandBCGS2, 1 BCGS-PIP)
  Mat Qbar, qs, T, C1;
  int cols = 0;
  TwoStageBigPanel(const Mat& Q_, const Sketch* S_, int K_, int pip_);
  Mat add_panel(const Mat& Vj);
  // QB, R_{Q,B}, R_BB and the coordinates of Qbar_B in [Q, Q_B]
  void finish(Mat& QB, Mat& RQB, Mat& RBB, Mat& coords);
};

OrthResult block_orth_two_stage(const Mat& V, int s, int s_hat, const Sketch* S, bool v0, int pip);

}  // namespace oracle

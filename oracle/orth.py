"""Block orthogonalization schemes, written step by step (oracle; test infrastructure).

The paper's pseudocode figures are not part of its text, so every scheme below
is restated from the prose; each function cites the passage it follows.

Conventions: V is n x c (float64).  The result is Q (n x c, Q^T Q = I) and R
(c x c upper triangular, non-negative diagonal) with V = QR (Figure 1 caption).
``v0=True`` means column 0 is the single starting vector V_0 = [v_0] (Table 1),
which is normalised (CholQR of one column) before the blocks of ``s`` columns.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dense import cholesky_upper, householder_qr, solve_right_upper
from .sketch import Sketch


class Breakdown(Exception):
    """A Cholesky factorisation met a non-positive pivot (Section 5.1)."""

    def __init__(self, column: int, block: int = -1, where: str = ""):
        super().__init__(f"Cholesky breakdown at column {column} (block {block}, {where})")
        self.column = column
        self.block = block
        self.where = where


# --- Figure 2a: BCGS -------------------------------------------------------------
def bcgs(Q: np.ndarray, W: np.ndarray):
    """C = Q^T W;  W_hat = W - Q C   (Section 9 lists these two operations)."""
    if Q.shape[1] == 0:
        return np.zeros((0, W.shape[1])), W.copy()
    C = Q.T @ W
    return C, W - Q @ C


# --- Figure 2b: CholQR -----------------------------------------------------------
def cholqr(W: np.ndarray, where: str = "cholqr"):
    """G = W^T W; R = chol(G) (upper, G = R^T R); Q = W R^{-1}  (Section 5.1)."""
    G = W.T @ W
    R, info = cholesky_upper(G)
    if info >= 0:
        raise Breakdown(info, where=where)
    return solve_right_upper(W, R), R


def cholqr2(W: np.ndarray):
    """CholQR twice: [Q1,R1]=CholQR(W); [Q,R2]=CholQR(Q1); R = R2 R1 (Section 5.1)."""
    Q1, R1 = cholqr(W, where="cholqr2-first")
    Q, R2 = cholqr(Q1, where="cholqr2-second")
    return Q, R2 @ R1


# --- Figure 4a: RandHH, Figure 4b: RandCholQR ------------------------------------
def rand_hh(W: np.ndarray, sketch: Sketch):
    """w = S W (sketch); R_hat = R of Householder QR(w); Q_bar = W R_hat^{-1} (Section 5.2)."""
    w = sketch.apply(W)
    Rh = householder_qr(w)
    return solve_right_upper(W, Rh), Rh


def rand_cholqr(W: np.ndarray, sketch: Sketch):
    """RandHH then CholQR of Q_bar; R = R' R_hat (Section 5.2, Proposition 5.2)."""
    Qbar, Rh = rand_hh(W, sketch)
    Qh, Rp = cholqr(Qbar, where="randcholqr")
    return Qh, Rp @ Rh


# --- Figure 2c: BCGS2 with a first intra-block step ------------------------------
def bcgs2_block(Q: np.ndarray, Vj: np.ndarray, intra):
    """One block of BCGS2 (Section 4; Barlow's BCGSI+ structure):

    [C1, W]     = BCGS(Q, V_j)
    [Qh, Rh]    = IntraBlk(W)            (RandCholQR, or CholQR2 for the baseline)
    [C2, Wt]    = BCGS(Q, Qh)
    [Q_j, R2]   = CholQR(Wt)
    R_{Q,j} = C1 + C2 Rh,   R_jj = R2 Rh.
    """
    C1, W = bcgs(Q, Vj)
    Qh, Rh = intra(W)
    C2, Wt = bcgs(Q, Qh)
    Qj, R2 = cholqr(Wt, where="final-cholqr")
    return Qj, C1 + C2 @ Rh, R2 @ Rh


@dataclass
class OrthResult:
    Q: np.ndarray
    R: np.ndarray
    ok: bool = True
    breakdown_block: int = -1
    breakdown_column: int = -1
    breakdown_where: str = ""
    extra: dict = field(default_factory=dict)


def _start(V: np.ndarray, v0: bool):
    n, c = V.shape
    Q = np.zeros((n, c))
    R = np.zeros((c, c))
    p = 0
    if v0:
        q, r = cholqr(V[:, :1], where="v0")
        Q[:, :1] = q
        R[0, 0] = r[0, 0]
        p = 1
    return Q, R, p


def block_orth_one_stage(V: np.ndarray, s: int, sketch: Sketch | None, intra: str = "rand",
                         v0: bool = False) -> OrthResult:
    """One-stage BCGS2 over blocks of ``s`` columns (Section 5).

    intra = "rand": RandCholQR first intra-block step (Figure 4b).
    intra = "cholqr2": CholQR2 first intra-block step (the deterministic baseline).
    A Cholesky breakdown stops the scheme and is reported with its block index
    (0-based over the blocks of s columns) and column within the block.
    """
    V = np.asarray(V, dtype=np.float64)
    n, c = V.shape
    Q, R, p = _start(V, v0)
    if (c - p) % s != 0:
        raise ValueError("number of columns after v0 must be a multiple of s")
    if intra == "rand":
        intra_fn = lambda W: rand_cholqr(W, sketch)  # noqa: E731
    elif intra == "cholqr2":
        intra_fn = cholqr2
    else:
        raise ValueError(intra)
    blk = 0
    while p < c:
        try:
            Qj, Rtop, Rjj = bcgs2_block(Q[:, :p], V[:, p:p + s], intra_fn)
        except Breakdown as e:
            return OrthResult(Q, R, False, blk, e.column, e.where)
        Q[:, p:p + s] = Qj
        R[:p, p:p + s] = Rtop
        R[p:p + s, p:p + s] = Rjj
        p += s
        blk += 1
    return OrthResult(Q, R)


# --- Figures 5-7: two-stage with RandBCGS2 preprocessing --------------------------
def sketched_bcgs2_hh(qs: np.ndarray, v: np.ndarray):
    """BCGS2 with Householder intra-block step on sketched vectors (Section 7.2).

    qs: d x p' sketched orthonormal basis of the earlier panels of the big panel;
    v : d x k sketch of the new panel.  Returns (q_new, T_col, T_jj) with
    v = qs T_col + q_new T_jj and [qs, q_new] orthonormal.
    """
    if qs.shape[1] == 0:
        qn, Tjj = householder_qr(v, want_q=True)
        return qn, np.zeros((0, v.shape[1])), Tjj
    c1 = qs.T @ v
    v1 = v - qs @ c1
    c2 = qs.T @ v1
    v2 = v1 - qs @ c2
    qn, Tjj = householder_qr(v2, want_q=True)
    return qn, c1 + c2, Tjj


def bcgs_pip(Qbar: np.ndarray, Vh: np.ndarray):
    """BCGS with the Pythagorean inner product (Section 7.1): one reduction of
    [Qbar, Vh]^T Vh gives P = Qbar^T Vh and G = Vh^T Vh; the Pythagorean rule
    replaces the Gram of the projected block by G - P^T P, whose Cholesky factor is
    T_jj; then Qbar_j = (Vh - Qbar P) T_jj^{-1}.  With no earlier panel it is CholQR
    (the section's footnote).  Returns (Qbar_j, T_col = P, T_jj)."""
    P = Qbar.T @ Vh
    G = Vh.T @ Vh
    Tjj, info = cholesky_upper(G - P.T @ P)
    if info >= 0:
        raise Breakdown(info, where="bcgs-pip")
    return solve_right_upper(Vh - Qbar @ P, Tjj), P, Tjj


class TwoStageBigPanel:
    """State of one big panel of the two-stage scheme (Sections 6-7).

    Per panel j (``add_panel``):
      [C1_j, Vh_j] = BCGS(Q, V_j)                     (inter big-panel BCGS)
      preprocessing, preproc = "rand" (RandBCGS2, Section 7.2):
        v_j = S Vh_j                                   (sketch)
        [q_j, T_{<j,j}, T_jj] = sketched BCGS2-HH(qs, v_j)
        Qbar_j = (Vh_j - Qbar_{<j} T_{<j,j}) T_jj^{-1} (forward substitution,
                                                       Appendix: Qbar = Vh T^{-1})
      preproc = "pip" (BCGS-PIP, Section 7.1): [Qbar_j, T_{<j,j}, T_jj] =
        BCGS-PIP(Qbar_{<j}, Vh_j)
    At the end (``finish``):
      [Qh_B, R'] = CholQR(Qbar_B);  [C2, Wt] = BCGS(Q, Qh_B);  [Q_B, R2] = CholQR(Wt)
      R_{Q,B} = C1 + C2 R' T,  R_BB = R2 R' T.
    ``coords_qbar`` = the coordinates of Qbar_B in [Q, Q_B]: [C2 R'; R2 R'].
    """

    def __init__(self, Q: np.ndarray, sketch: Sketch | None, K: int, preproc: str = "rand"):
        if preproc not in ("rand", "pip"):
            raise ValueError("preproc must be 'rand' or 'pip'")
        self.Q = Q
        self.sketch = sketch
        self.preproc = preproc
        self.K = K
        n = Q.shape[0]
        self.Qbar = np.zeros((n, 0))
        self.qs = np.zeros((sketch.d if sketch is not None else 0, 0))
        self.T = np.zeros((K, K))
        self.C1 = np.zeros((Q.shape[1], K))
        self.cols = 0

    def add_panel(self, Vj: np.ndarray) -> np.ndarray:
        k = Vj.shape[1]
        a = self.cols
        C1, Vh = bcgs(self.Q, Vj)
        self.C1[:, a:a + k] = C1
        if self.preproc == "pip":
            Qbj, Tcol, Tjj = bcgs_pip(self.Qbar, Vh)
            self.T[:a, a:a + k] = Tcol
            self.T[a:a + k, a:a + k] = Tjj
            self.Qbar = np.hstack([self.Qbar, Qbj])
            self.cols += k
            return Qbj
        v = self.sketch.apply(Vh)
        qn, Tcol, Tjj = sketched_bcgs2_hh(self.qs, v)
        self.T[:a, a:a + k] = Tcol
        self.T[a:a + k, a:a + k] = Tjj
        Qbj = solve_right_upper(Vh - self.Qbar @ Tcol, Tjj)
        self.Qbar = np.hstack([self.Qbar, Qbj])
        self.qs = np.hstack([self.qs, qn])
        self.cols += k
        return Qbj

    def finish(self):
        K = self.cols
        T = self.T[:K, :K]
        Qh, Rp = cholqr(self.Qbar, where="bigpanel-cholqr")
        C2, Wt = bcgs(self.Q, Qh)
        QB, R2 = cholqr(Wt, where="bigpanel-final-cholqr")
        RQB = self.C1[:, :K] + C2 @ Rp @ T
        RBB = R2 @ Rp @ T
        coords_qbar = np.vstack([C2 @ Rp, R2 @ Rp])
        return QB, RQB, RBB, coords_qbar


def block_orth_two_stage(V: np.ndarray, s: int, s_hat: int, sketch: Sketch | None,
                         v0: bool = False, preproc: str = "rand") -> OrthResult:
    """Two-stage block orthogonalization (flat form, Figure 6 / Section 6): big panels
    of ``s_hat`` columns made of panels of ``s``, preprocessed by RandBCGS2
    (preproc="rand", Section 7.2) or BCGS-PIP (preproc="pip", Section 7.1)."""
    V = np.asarray(V, dtype=np.float64)
    n, c = V.shape
    Q, R, p = _start(V, v0)
    if (c - p) % s_hat != 0 or s_hat % s != 0:
        raise ValueError("columns after v0 must be a multiple of s_hat, and s_hat of s")
    big = 0
    while p < c:
        bp = TwoStageBigPanel(Q[:, :p], sketch, s_hat, preproc)
        try:
            for j in range(s_hat // s):
                bp.add_panel(V[:, p + j * s:p + (j + 1) * s])
            QB, RQB, RBB, _ = bp.finish()
        except Breakdown as e:
            return OrthResult(Q, R, False, big, e.column, e.where)
        Q[:, p:p + s_hat] = QB
        R[:p, p:p + s_hat] = RQB
        R[p:p + s_hat, p:p + s_hat] = RBB
        p += s_hat
        big += 1
    return OrthResult(Q, R)


def block_orth_cholqr2(V: np.ndarray, s: int, v0: bool = False) -> OrthResult:
    """BCGS2 with CholQR2 as the first intra-block step (the baseline of Figure 4)."""
    return block_orth_one_stage(V, s, None, intra="cholqr2", v0=v0)


def householder_reference(V: np.ndarray):
    """The exact-result reference: Householder QR of all of V, R with diag >= 0.
    For full-rank V the QR factorisation with non-negative diagonal is unique, so
    every stable scheme approximates this Q and R."""
    return householder_qr(V, want_q=True)

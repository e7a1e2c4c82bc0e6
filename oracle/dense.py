"""Small dense kernels of the oracle (test infrastructure).

* ``cholesky_upper``: G = R^T R with R upper triangular, computed column by
  column; the first pivot that is not positive (or not finite) is reported as a
  breakdown, the failure mode of CholQR that Section 5.1 and the caption of
  Figure 4 describe ("failed with non-positive pivots").
* ``householder_qr``: Householder QR (Golub and Van Loan, Algorithm 5.2.1)
  written out, returning R with a non-negative diagonal (the normalisation of
  the QR factorisation in the caption of Figure 1) and optionally the thin Q.
* ``solve_right_upper``: X = W R^{-1} (the TRSM of CholQR and RandHH).
* ``gram``: C = X^T Y, the reduction of BCGS and CholQR, with products and sums in
  numpy's extended ``longdouble`` type (the reference for Gram kernels).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def cholesky_upper(G: np.ndarray):
    """Return (R, info): info = -1 on success, else the 0-based column of the
    first non-positive or non-finite pivot (R is then only valid above it)."""
    G = np.asarray(G, dtype=np.float64)
    k = G.shape[0]
    R = np.zeros((k, k))
    for j in range(k):
        piv = G[j, j] - np.dot(R[:j, j], R[:j, j])
        if not np.isfinite(piv) or piv <= 0.0:
            return R, j
        rjj = np.sqrt(piv)
        R[j, j] = rjj
        if j + 1 < k:
            R[j, j + 1:] = (G[j, j + 1:] - R[:j, j] @ R[:j, j + 1:]) / rjj
    return R, -1


def householder_qr(A: np.ndarray, want_q: bool = False):
    """Householder QR of an m x k matrix (m >= k); R has a non-negative diagonal."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, k = A.shape
    if m < k:
        raise ValueError("householder_qr needs m >= k")
    vs = []
    betas = []
    for j in range(k):
        x = A[j:, j]
        alpha = np.linalg.norm(x)
        v = x.copy()
        if alpha == 0.0:
            vs.append(None)
            betas.append(0.0)
            continue
        # reflect x onto -sign(x0) * alpha * e1 (no cancellation in v0)
        s = 1.0 if x[0] >= 0 else -1.0
        v[0] = x[0] + s * alpha
        beta = 2.0 / np.dot(v, v)
        A[j:, j:] -= beta * np.outer(v, v @ A[j:, j:])
        vs.append(v)
        betas.append(beta)
    R = np.triu(A[:k, :k])
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    R = sgn[:, None] * R
    if not want_q:
        return R
    Q = np.zeros((m, k))
    Q[:k, :k] = np.eye(k)
    for j in range(k - 1, -1, -1):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= betas[j] * np.outer(v, v @ Q[j:, :])
    Q = Q * sgn
    return Q, R


def solve_right_upper(W: np.ndarray, R: np.ndarray) -> np.ndarray:
    """X = W R^{-1} for upper-triangular R (rows of W solved independently)."""
    W = np.asarray(W, dtype=np.float64)
    if W.shape[1] == 0:
        return W.copy()
    # X R = W  <=>  R^T X^T = W^T
    return sla.solve_triangular(R, W.T, trans="T", lower=False).T


def gram(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """C = X^T Y (Section 9 lists it as the reduction of BCGS, C = Q^T W, and of
    CholQR, G = W^T W).  Products and sums in extended precision (longdouble), rounded
    to float64 once, so its own error is far below float64 rounding."""
    Xl = np.asarray(X, dtype=np.longdouble)
    Yl = np.asarray(Y, dtype=np.longdouble)
    return (Xl.T @ Yl).astype(np.float64)

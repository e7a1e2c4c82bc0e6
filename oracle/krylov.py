"""CSR SpMV, monomial matrix-powers kernel and s-step GMRES (oracle; test infrastructure).

s-step GMRES (Section 4, Figure 1), right-preconditioned: the iteration works
on y with x = M^{-1} y and the operator Ahat = A M^{-1}.  For the Jacobi
preconditioner M = diag(A), so Ahat is A with its columns divided by the
diagonal.  Readings of points the paper leaves open (its pseudocode figure is
not in the text):

* Start: r = b - Ahat y, beta = ||r||, q_0 = r / beta (the V_0 = [v_0] block).
* Panel: the matrix-powers kernel applies Ahat s times to the panel's start
  vector u (monomial basis): V_j = [Ahat u, Ahat^2 u, ..., Ahat^s u].  One-stage:
  u is the last orthonormal basis vector.  Two-stage: u is the last
  preprocessed vector qbar of the previous panel inside a big panel, and the
  last final basis vector at a big-panel boundary (the paper notes, Section 8,
  that the start vector is preprocessed before the next panel is generated).
* Hessenberg: with U the generators and W = Ahat U the MPK outputs written in
  the orthonormal basis as U = Q X (X upper triangular) and W = Q Y, the Arnoldi
  relation Ahat Q = Q H gives H = Y X^{-1}.
* Least squares min ||beta e_1 - H z|| after every panel (one-stage) or big
  panel (two-stage); when the estimate falls to tol * ||b||, or the restart
  length m is reached, y += Q z and the cycle restarts from the true residual.
* Convergence is declared on the true relative residual ||b - A x|| / ||b||.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .dense import solve_right_upper
from .orth import Breakdown, TwoStageBigPanel, bcgs2_block, cholqr, cholqr2, rand_cholqr
from .sketch import Sketch


def spmv(A, x: np.ndarray) -> np.ndarray:
    """y = A x for a CSR matrix (anything with rowptr/col/val or a scipy matrix)."""
    M = A.to_scipy() if hasattr(A, "to_scipy") else A
    return M @ x


def mpk(Ahat, u: np.ndarray, s: int) -> np.ndarray:
    """Monomial matrix-powers kernel: [Ahat u, Ahat^2 u, ..., Ahat^s u] (Section 4)."""
    V = np.empty((u.shape[0], s))
    v = u
    for i in range(s):
        v = Ahat @ v
        V[:, i] = v
    return V


def jacobi_scaled(A):
    """Return (Ahat = A D^{-1}, dinv) for the right Jacobi preconditioner M = D = diag(A)."""
    M = A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)
    diag = M.diagonal()
    if np.any(diag == 0):
        raise ValueError("Jacobi preconditioner needs a nonzero diagonal")
    dinv = 1.0 / diag
    return (M @ sp.diags(dinv)).tocsr(), dinv


@dataclass
class GmresResult:
    x: np.ndarray
    converged: bool
    iterations: int
    restarts: int
    relres: float
    history: list = field(default_factory=list)       # (iterations, true relative residual)
    estimates: list = field(default_factory=list)     # (iterations, estimated relative residual)
    breakdown: str = ""


def _ls(H: np.ndarray, beta: float):
    g = np.zeros(H.shape[0])
    g[0] = beta
    z = np.linalg.lstsq(H, g, rcond=None)[0]
    return z, float(np.linalg.norm(g - H @ z))


def sstep_gmres(A, b, x0=None, *, s: int, m: int, tol: float, s_hat: int | None = None,
                scheme: str = "one", intra: str = "rand", max_restarts: int = 200,
                d: int | None = None, zeta: int = 8, seed: int = 42,
                precond: str = "jacobi", preproc: str = "rand") -> GmresResult:
    """s-step GMRES(m) with one-stage (RandCholQR or CholQR2 BCGS2) or two-stage
    (big panels of s_hat, preprocessed by RandBCGS2 or BCGS-PIP) block
    orthogonalization."""
    if precond == "jacobi":
        Ahat, dinv = jacobi_scaled(A)
    else:
        Ahat = (A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)).tocsr()
        dinv = np.ones(Ahat.shape[0])
    n = Ahat.shape[0]
    if m % s != 0:
        raise ValueError("m must be a multiple of s")
    if scheme == "two":
        s_hat = s_hat or m
        if m % s_hat != 0 or s_hat % s != 0:
            raise ValueError("need s | s_hat | m")
    d = d or 4 * (m + 1)
    sketch = Sketch(n, d, zeta, seed)
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    y = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64) / dinv
    its = 0
    res = GmresResult(x=dinv * y, converged=False, iterations=0, restarts=0, relres=np.inf)
    if intra == "rand":
        intra_fn = lambda W: rand_cholqr(W, sketch)  # noqa: E731
    else:
        intra_fn = cholqr2
    for cycle in range(max_restarts + 1):
        r = b - Ahat @ y
        try:
            q0, r00 = cholqr(r[:, None], where="v0")
        except Breakdown:
            res.converged = True  # r == 0
            res.relres = 0.0
            break
        beta = float(r00[0, 0])
        rel = beta / bnorm
        res.history.append((its, rel))
        res.relres = rel
        if rel <= tol:
            res.converged = True
            break
        if cycle == max_restarts:
            break
        res.restarts = cycle
        Qb = np.zeros((n, m + 1))
        Qb[:, 0] = q0[:, 0]
        R = np.zeros((m + 1, m + 1))
        R[0, 0] = beta
        X = np.zeros((m, m))
        Y = np.zeros((m + 1, m))
        ncols = 1
        z = np.zeros(0)
        try:
            while ncols < m + 1:
                P = ncols
                if scheme == "one":
                    V = mpk(Ahat, Qb[:, P - 1], s)
                    Qj, Rtop, Rjj = bcgs2_block(Qb[:, :P], V, intra_fn)
                    Qb[:, P:P + s] = Qj
                    R[:P, P:P + s] = Rtop
                    R[P:P + s, P:P + s] = Rjj
                    X[P - 1, P - 1] = 1.0
                    for i in range(1, s):
                        X[:P + i, P - 1 + i] = R[:P + i, P + i - 1]
                    Y[:P + s, P - 1:P - 1 + s] = R[:P + s, P:P + s]
                    ncols += s
                    its += s
                else:
                    bp = TwoStageBigPanel(Qb[:, :P], sketch, s_hat, preproc)
                    gens = []
                    for j in range(s_hat // s):
                        if j == 0:
                            u = Qb[:, P - 1]
                            gens.append(None)
                        else:
                            u = bp.Qbar[:, -1]
                            gens.append(bp.cols - 1)
                        bp.add_panel(mpk(Ahat, u, s))
                    QB, RQB, RBB, cq = bp.finish()
                    Qb[:, P:P + s_hat] = QB
                    R[:P, P:P + s_hat] = RQB
                    R[P:P + s_hat, P:P + s_hat] = RBB
                    for j, g in enumerate(gens):
                        c = P + j * s
                        if g is None:
                            X[c - 1, c - 1] = 1.0
                        else:
                            X[:P + g + 1, c - 1] = cq[:P + g + 1, g]
                        for i in range(1, s):
                            X[:c + i, c - 1 + i] = R[:c + i, c + i - 1]
                    Y[:P + s_hat, P - 1:P - 1 + s_hat] = R[:P + s_hat, P:P + s_hat]
                    ncols += s_hat
                    its += s_hat
                k = ncols - 1
                H = solve_right_upper(Y[:ncols, :k], X[:k, :k])
                z, est = _ls(H, beta)
                res.estimates.append((its, est / bnorm))
                if est / bnorm <= tol:
                    break
        except Breakdown as e:
            res.breakdown = str(e)
            res.iterations = its
            res.x = dinv * y
            return res
        k = ncols - 1
        y = y + Qb[:, :k] @ z
    res.iterations = its
    res.x = dinv * y
    return res


def householder_gmres(A, b, x0=None, *, m: int, tol: float, max_restarts: int = 200,
                      precond: str = "jacobi") -> GmresResult:
    """GMRES(m) with Householder-reflector Arnoldi (Walker, SISC 1988), the most
    stable formulation; used as the brute-force reference for small n."""
    if precond == "jacobi":
        Ahat, dinv = jacobi_scaled(A)
    else:
        Ahat = (A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)).tocsr()
        dinv = np.ones(Ahat.shape[0])
    n = Ahat.shape[0]
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    y = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64) / dinv
    res = GmresResult(x=dinv * y, converged=False, iterations=0, restarts=0, relres=np.inf)
    its = 0
    for cycle in range(max_restarts + 1):
        r = b - Ahat @ y
        beta = float(np.linalg.norm(r))
        rel = beta / bnorm
        res.history.append((its, rel))
        res.relres = rel
        if rel <= tol:
            res.converged = True
            break
        if cycle == max_restarts:
            break
        res.restarts = cycle
        W = []
        H = np.zeros((m + 1, m))
        zv = r.copy()
        g0 = 0.0
        kdone = 0
        z = np.zeros(0)
        for j in range(m + 1):
            w = zv.copy()
            w[:j] = 0.0
            alpha = np.linalg.norm(w[j:])
            if alpha == 0.0:
                break
            sgn = 1.0 if w[j] >= 0 else -1.0
            w[j] += sgn * alpha
            w /= np.linalg.norm(w)
            W.append(w)
            h = zv - 2.0 * w * (w @ zv)
            if j == 0:
                g0 = h[0]
            else:
                H[:j + 1, j - 1] = h[:j + 1]
                kdone = j
                g = np.zeros(j + 1)
                g[0] = g0
                z = np.linalg.lstsq(H[:j + 1, :j], g, rcond=None)[0]
                est = float(np.linalg.norm(g - H[:j + 1, :j] @ z))
                its += 1
                res.estimates.append((its, est / bnorm))
                if est / bnorm <= tol:
                    break
            if j == m:
                break
            q = np.zeros(n)
            q[j] = 1.0
            for i in range(j, -1, -1):
                q -= 2.0 * W[i] * (W[i] @ q)
            zv = Ahat @ q
            for i in range(j + 1):
                zv -= 2.0 * W[i] * (W[i] @ zv)
        upd = np.zeros(n)
        for i in range(kdone):
            q = np.zeros(n)
            q[i] = 1.0
            for t in range(i, -1, -1):
                q -= 2.0 * W[t] * (W[t] @ q)
            upd += z[i] * q
        y = y + upd
    res.iterations = its
    res.x = dinv * y
    return res

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


# --- Newton basis (Section 4 mentions it as the MPK option of Trilinos; Bai, Hu and
# Reichel, IMA J. Numer. Anal. 14, 1994) ------------------------------------------
def leja_order(theta: np.ndarray, rtol: float = 1e-12) -> list:
    """Modified Leja ordering of the Ritz values ``theta``: the first point has the
    largest modulus, every next point maximises the product of its distances to the
    points already chosen (sum of logarithms), and a complex point is followed at once
    by its conjugate.  Values whose imaginary part is below rtol*|value| count as real."""
    theta = np.asarray(theta, dtype=np.complex128)
    scale = max(float(np.abs(theta).max()), 1e-300) if theta.size else 1.0
    cand = []
    for z in theta:
        if abs(z.imag) <= rtol * scale:
            cand.append(complex(z.real, 0.0))
        elif z.imag > 0:
            cand.append(complex(z))
    out = []
    while cand:
        if not out:
            j = int(np.argmax([abs(z) for z in cand]))
        else:
            def score(z):
                return sum(np.log(max(abs(z - w), 1e-300 * scale)) for w in out)
            j = int(np.argmax([score(z) for z in cand]))
        z = cand.pop(j)
        out.append(z)
        if z.imag != 0.0:
            out.append(z.conjugate())
    return out


def newton_shifts(H: np.ndarray, s: int):
    """Shifts for s Newton-basis vectors from the square upper-Hessenberg H (the
    last cycle's Arnoldi matrix): the first s of the Ritz values in Leja order, as
    the real recurrence v_{i+1} = (Ahat - alpha_i) v_i + beta_i v_{i-1}, with
    alpha_i = Re theta_i and beta_i = (Im theta_i)^2 for the second value of a
    conjugate pair (0 otherwise).  A pair split by the s-th position contributes
    its real part only."""
    order = leja_order(np.linalg.eigvals(H))
    alpha, beta = np.zeros(s), np.zeros(s)
    i = 0
    while i < s and i < len(order):
        z = order[i]
        alpha[i] = z.real
        if z.imag > 0 and i + 1 < s:
            alpha[i + 1] = z.real
            beta[i + 1] = z.imag ** 2
            i += 2
        else:
            i += 1
    return alpha, beta


# --- Chebyshev basis (Sections 5 and 8 name it beside the Newton basis; Joubert and
# Carey, Comput. Math. Appl. 24, 1992) ---------------------------------------------
def chebyshev_ellipse(theta: np.ndarray):
    """Ellipse enclosing the Ritz values ``theta`` (closed under conjugation), with its
    centre c on the real axis at the midpoint of their real extent and its axes along
    the real and imaginary directions: among those, the one of smallest capacity
    (a + b)/2 (a, b the real and imaginary semi-axes).  For a real semi-axis a the
    smallest enclosing b is b(a) = max_i y_i a / sqrt(a^2 - dx_i^2) (dx_i = Re theta_i - c,
    y_i = |Im theta_i|); a + b(a) is convex on a > a0 (a0 half the real extent), so a is
    found by bisection on the sign of its right derivative
    1 - y_i dx_i^2 / (a^2 - dx_i^2)^(3/2) (i the maximising value).  Real values give
    the interval [min, max] itself (b = 0); values on one vertical line give the
    segment (a = 0).  Returns (c, a, b)."""
    theta = np.asarray(theta, dtype=np.complex128)
    x, y = theta.real, np.abs(theta.imag)
    c = 0.5 * (float(x.max()) + float(x.min()))
    a0 = 0.5 * (float(x.max()) - float(x.min()))
    b0 = float(y.max())
    if b0 == 0.0:
        return c, a0, 0.0
    if a0 == 0.0:
        return c, 0.0, b0
    dx, y = (x - c)[y > 0], y[y > 0]

    def b_and_slope(a):
        r = a * a - dx * dx
        g = y * a / np.sqrt(r)
        i = int(np.argmax(g))
        return float(g[i]), 1.0 - y[i] * dx[i] ** 2 / r[i] ** 1.5

    # the minimiser a* satisfies a* <= a* + b(a*) <= a1 + b(a1) for any a1 > a0
    a1 = 2.0 * a0 + b0
    lo, hi = a0, a1 + b_and_slope(a1)[0]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if b_and_slope(mid)[1] < 0.0:
            lo = mid
        else:
            hi = mid
    return c, hi, b_and_slope(hi)[0]


def chebyshev_shifts(H: np.ndarray, s: int):
    """Recurrence of s Chebyshev-basis vectors for the ellipse (c, a, b) enclosing the
    eigenvalues of the square upper-Hessenberg H (``chebyshev_ellipse``), with
    e2 = a^2 - b^2 its squared half focal distance: p_k(z) = 2 (e/2)^k T_k((z - c)/e),
    k >= 1 (T_k the Chebyshev polynomials of the first kind), which satisfy
    p_1 = (z - c), p_2 = (z - c) p_1 - (e2/2), p_{k+1} = (z - c) p_k - (e2/4) p_{k-1};
    in the form v_{i+1} = (Ahat - alpha_i) v_i + beta_i v_{i-1}: alpha_i = c,
    beta_0 = 0, beta_1 = -e2/2, beta_i = -e2/4 (i >= 2)."""
    c, a, b = chebyshev_ellipse(np.linalg.eigvals(H))
    e2 = a * a - b * b
    alpha = np.full(s, c)
    beta = np.full(s, -0.25 * e2)
    beta[0] = 0.0
    if s > 1:
        beta[1] = -0.5 * e2
    return alpha, beta


def mpk_newton(Ahat, u: np.ndarray, alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Newton matrix-powers kernel: v_0 = u, v_{i+1} = (Ahat - alpha_i) v_i + beta_i v_{i-1}
    (beta_0 = 0); returns [v_1, ..., v_s].  alpha = beta = 0 is the monomial basis."""
    s = len(alpha)
    V = np.empty((u.shape[0], s))
    prev, v = None, u
    for i in range(s):
        w = Ahat @ v - alpha[i] * v
        if beta[i] != 0.0:
            w = w + beta[i] * prev
        V[:, i] = w
        prev, v = v, w
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
                precond: str = "jacobi", preproc: str = "rand",
                basis: str = "monomial") -> GmresResult:
    """s-step GMRES(m) with one-stage (RandCholQR or CholQR2 BCGS2) or two-stage
    (big panels of s_hat, preprocessed by RandBCGS2 or BCGS-PIP) block
    orthogonalization.  basis = "newton" / "chebyshev": the first cycle is standard
    GMRES (panels of one column), later cycles use the Newton basis with shifts from
    the first cycle's Ritz values, or the Chebyshev basis of the ellipse enclosing
    them;
    since Ahat U = W + U B for the generators U of a panel (B bidiagonal with
    alpha on the diagonal and -beta above it; the Chebyshev basis is the same
    three-term form), the Hessenberg matrix becomes
    (Y + X B) X^{-1}."""
    if basis not in ("monomial", "newton", "chebyshev"):
        raise ValueError(f"unknown basis {basis!r}")
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
    alpha, beta_s = np.zeros(s), np.zeros(s)   # monomial until shifts are known

    def gen(u, k):
        return mpk_newton(Ahat, u, alpha[:k], beta_s[:k])

    def shift_columns(Y, X, c0, k):
        # Y(:, c0 + i) += alpha_i X(:, c0 + i) - beta_i X(:, c0 + i - 1)
        for i in range(k):
            Y[:m, c0 + i] += alpha[i] * X[:, c0 + i]
            if beta_s[i] != 0.0:
                Y[:m, c0 + i] -= beta_s[i] * X[:, c0 + i - 1]

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
        # Newton basis: the cycle that provides the Ritz values is standard GMRES
        # (panels of one column, one-stage)
        sc = 1 if (basis != "monomial" and cycle == 0) else s
        try:
            while ncols < m + 1:
                P = ncols
                if scheme == "one" or sc != s:
                    V = gen(Qb[:, P - 1], sc)
                    Qj, Rtop, Rjj = bcgs2_block(Qb[:, :P], V, intra_fn)
                    Qb[:, P:P + sc] = Qj
                    R[:P, P:P + sc] = Rtop
                    R[P:P + sc, P:P + sc] = Rjj
                    X[P - 1, P - 1] = 1.0
                    for i in range(1, sc):
                        X[:P + i, P - 1 + i] = R[:P + i, P + i - 1]
                    Y[:P + sc, P - 1:P - 1 + sc] = R[:P + sc, P:P + sc]
                    shift_columns(Y, X, P - 1, sc)
                    ncols += sc
                    its += sc
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
                        bp.add_panel(gen(u, s))
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
                    for j in range(len(gens)):
                        shift_columns(Y, X, P - 1 + j * s, s)
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
        if basis == "newton" and cycle == 0:
            alpha, beta_s = newton_shifts(H[:k, :k], s)
        elif basis == "chebyshev" and cycle == 0:
            alpha, beta_s = chebyshev_shifts(H[:k, :k], s)
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

"""Learned sparse-approximate-inverse preconditioner: graph network, loss and the
classical SPAI (oracle; test infrastructure).

Not in the paper: the workload asks for a small graph network that maps a
matrix's entries to the values of a right preconditioner M on A's own sparsity
pattern, so that the matrix-powers kernel stays linear (v_{k+1} = A M v_k) and
s-step GMRES stays valid.  This module is the float64 reference of that network,
of its loss and gradient, and of the classical SPAI minimiser used as a pin.

Graph: nodes are the rows of A; every stored entry (i, j) of A (diagonal
included) is an edge carrying a message from node j to node i.  With D = diag(A)
and Ahat = D^{-1} A:

  node features  f_i  = [sum_{j != i} |Ahat_ij|, sum_{j != i} |Ahat_ji|]
  edge features  x_ij = [Ahat_ij, Ahat_ji (0 if (j, i) is not stored), [i == j]]
  h0 = relu(Wn f + bn)                  (width 32)
  e0 = relu(We x + be)                  (width 32)
  3 layers:  m_ij = relu(Wm [e_ij; h_j] + bm)
             agg_i = sum_j m_ij
             h_i  <- h_i + relu(Wh [h_i; agg_i] + bh)
             e_ij <- e_ij + m_ij
  out_ij = wo . [e_ij; h_i; h_j] + bo + [i == j]
  M_ij = out_ij / A_ii

With all weights zero, M = D^{-1} (Jacobi).  Loss over residual vectors r
(columns of Rb):  L = mean_k ||r_k - A M r_k||^2 / ||r_k||^2.  Over all unit
vectors r this is ||I - A M||_F^2 / n, whose minimiser on pattern(A) is the
classical SPAI (Grote and Huckle, SISC 1997): column j of M solves
min ||e_j - A m_j|| with m_j supported on the pattern of column j.

Weights are rounded to bfloat16 before use (``to_bf16``), matching the
network's BF16 weights; activations and sums are float64 here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

WIDTH = 32
LAYERS = 3


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest even on the 16 dropped bits
    of the float32 encoding) and return them as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def param_shapes():
    """Names and shapes, in the flat order used by the library."""
    shapes = [("Wn", (WIDTH, 2)), ("bn", (WIDTH,)), ("We", (WIDTH, 3)), ("be", (WIDTH,))]
    for l in range(LAYERS):
        shapes += [(f"Wm{l}", (WIDTH, 2 * WIDTH)), (f"bm{l}", (WIDTH,)),
                   (f"Wh{l}", (WIDTH, 2 * WIDTH)), (f"bh{l}", (WIDTH,))]
    shapes += [("wo", (3 * WIDTH,)), ("bo", (1,))]
    return shapes


def n_params() -> int:
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unflatten(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in param_shapes():
        k = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return out


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def init_params(seed: int, scale: float = 0.5) -> np.ndarray:
    """He-like random initial weights, output layer zero (so the network starts at
    Jacobi)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes():
        if name.startswith("W"):
            p[name] = rng.standard_normal(shp) * scale * np.sqrt(2.0 / shp[1])
        else:
            p[name] = np.zeros(shp)
    return flatten(p)


class Graph:
    """Edge lists and features of a CSR matrix (float64)."""

    def __init__(self, A):
        M = A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)
        M = M.tocsr()
        M.sort_indices()
        self.A = M
        self.n = M.shape[0]
        self.row = np.repeat(np.arange(self.n), np.diff(M.indptr))
        self.col = M.indices.astype(np.int64)
        self.val = M.data.astype(np.float64)
        self.diag = M.diagonal()
        dinv = 1.0 / self.diag
        ah = self.val * dinv[self.row]                      # Ahat_ij
        # Ahat_ji for each stored (i, j): look up the transpose entry
        T = sp.csr_matrix((np.arange(1, len(self.val) + 1, dtype=np.float64), M.indices, M.indptr),
                          shape=M.shape)
        Tt = T.T.tocsr()
        # position of (j, i) in CSR order, 0 if absent
        pos = np.asarray(Tt[self.row, self.col]).ravel().astype(np.int64)
        aji = np.where(pos > 0, self.val[np.maximum(pos - 1, 0)], 0.0)
        ahT = aji * dinv[self.col]                          # Ahat_ji = a_ji / a_jj
        self.tpos = pos - 1                                  # -1 when absent
        off = self.row != self.col
        self.x = np.stack([ah, ahT, (~off).astype(np.float64)], axis=1)
        rs = np.bincount(self.row, weights=np.abs(ah) * off, minlength=self.n)
        cs = np.bincount(self.col, weights=np.abs(ah) * off, minlength=self.n)
        self.f = np.stack([rs, cs], axis=1)
        self.is_diag = (~off).astype(np.float64)


def _relu(x):
    return np.maximum(x, 0.0)


def forward(theta: np.ndarray, G: Graph, bf16: bool = True, keep: bool = False):
    """Return the values of M on A's pattern (CSR order) [and the saved activations]."""
    p = unflatten(theta)
    if bf16:
        p = {k: to_bf16(v) for k, v in p.items()}
    cache = {}
    zn = G.f @ p["Wn"].T + p["bn"]
    h = _relu(zn)
    ze = G.x @ p["We"].T + p["be"]
    e = _relu(ze)
    cache["zn"], cache["ze"] = zn, ze
    for l in range(LAYERS):
        u = np.concatenate([e, h[G.col]], axis=1)
        zm = u @ p[f"Wm{l}"].T + p[f"bm{l}"]
        m = _relu(zm)
        agg = np.zeros((G.n, WIDTH))
        np.add.at(agg, G.row, m)
        v = np.concatenate([h, agg], axis=1)
        zh = v @ p[f"Wh{l}"].T + p[f"bh{l}"]
        cache[f"u{l}"], cache[f"zm{l}"], cache[f"v{l}"], cache[f"zh{l}"] = u, zm, v, zh
        h = h + _relu(zh)
        e = e + m
    q = np.concatenate([e, h[G.row], h[G.col]], axis=1)
    out = q @ p["wo"] + p["bo"][0] + G.is_diag
    cache["q"] = q
    Mv = out / G.diag[G.row]
    if keep:
        return Mv, (p, cache)
    return Mv


def loss_and_dM(Mv: np.ndarray, G: Graph, Rb: np.ndarray):
    """Loss over residual columns Rb and its gradient w.r.t. the values of M."""
    Msp = sp.csr_matrix((Mv, G.col, G.A.indptr), shape=G.A.shape)
    Z = Msp @ Rb
    Y = G.A @ Z
    E = Rb - Y
    w = 1.0 / np.sum(Rb * Rb, axis=0)
    k = Rb.shape[1]
    L = float(np.sum(np.sum(E * E, axis=0) * w) / k)
    dY = -2.0 * E * w / k
    dZ = G.A.T @ dY
    dM = np.sum(dZ[G.row] * Rb[G.col], axis=1)
    return L, dM


def backward(theta: np.ndarray, G: Graph, dMv: np.ndarray, saved) -> np.ndarray:
    """Gradient of a scalar with respect to theta, given its gradient dMv w.r.t. the
    values of M (straight-through the bf16 rounding of the weights)."""
    p, cache = saved
    g = {k: np.zeros_like(v) for k, v in p.items()}
    dout = dMv / G.diag[G.row]
    q = cache["q"]
    g["wo"] = q.T @ dout
    g["bo"] = np.array([dout.sum()])
    dq = np.outer(dout, p["wo"])
    de = dq[:, :WIDTH].copy()
    dh = np.zeros((G.n, WIDTH))
    np.add.at(dh, G.row, dq[:, WIDTH:2 * WIDTH])
    np.add.at(dh, G.col, dq[:, 2 * WIDTH:])
    for l in reversed(range(LAYERS)):
        u, zm, v, zh = cache[f"u{l}"], cache[f"zm{l}"], cache[f"v{l}"], cache[f"zh{l}"]
        # h_{l+1} = h_l + relu(zh);  e_{l+1} = e_l + m
        dzh = dh * (zh > 0)
        g[f"Wh{l}"] += dzh.T @ v
        g[f"bh{l}"] += dzh.sum(axis=0)
        dv = dzh @ p[f"Wh{l}"]
        dh_l = dh + dv[:, :WIDTH]
        dagg = dv[:, WIDTH:]
        dm = de + dagg[G.row]
        dzm = dm * (zm > 0)
        g[f"Wm{l}"] += dzm.T @ u
        g[f"bm{l}"] += dzm.sum(axis=0)
        du = dzm @ p[f"Wm{l}"]
        de = de + du[:, :WIDTH]
        np.add.at(dh_l, G.col, du[:, WIDTH:])
        dh = dh_l
    dze = de * (cache["ze"] > 0)
    g["We"] = dze.T @ G.x
    g["be"] = dze.sum(axis=0)
    dzn = dh * (cache["zn"] > 0)
    g["Wn"] = dzn.T @ G.f
    g["bn"] = dzn.sum(axis=0)
    return flatten(g)


def loss_and_grad(theta: np.ndarray, G: Graph, Rb: np.ndarray, bf16: bool = True):
    Mv, saved = forward(theta, G, bf16=bf16, keep=True)
    L, dM = loss_and_dM(Mv, G, Rb)
    return L, backward(theta, G, dM, saved)


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015), bias-corrected; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def spai(A) -> np.ndarray:
    """Classical SPAI on A's pattern: column j of M minimises ||e_j - A m_j||_2 over
    vectors supported on the stored rows of column j of A (Grote and Huckle 1997).
    Returns M's values in A's CSR order."""
    G = Graph(A)
    Ac = G.A.tocsc()
    Ac.sort_indices()
    n = G.n
    Mcsc_vals = np.zeros(len(G.val))
    for j in range(n):
        J = Ac.indices[Ac.indptr[j]:Ac.indptr[j + 1]]      # support of column j of M
        sub = G.A[:, J]
        I = np.unique(sub.nonzero()[0])
        Ad = sub[I].toarray()
        rhs = (I == j).astype(np.float64)
        mj = np.linalg.lstsq(Ad, rhs, rcond=None)[0]
        Mcsc_vals[Ac.indptr[j]:Ac.indptr[j + 1]] = mj
    Mcsc = sp.csc_matrix((Mcsc_vals, Ac.indices, Ac.indptr), shape=G.A.shape).tocsr()
    Mcsc.sort_indices()
    # align to A's CSR pattern
    return np.asarray(Mcsc[G.row, G.col]).ravel()


def frobenius_loss(A, Mv) -> float:
    """||I - A M||_F^2 / n for M with values Mv on A's pattern."""
    G = Graph(A)
    Msp = sp.csr_matrix((Mv, G.col, G.A.indptr), shape=G.A.shape)
    R = sp.identity(G.n, format="csr") - G.A @ Msp
    return float(sp.linalg.norm(R, "fro") ** 2 / G.n)

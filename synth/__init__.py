"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module builds *inputs only*: test matrices V with prescribed per-block
condition numbers, sparse PDE matrices in CSR form, and right-hand sides.  It
holds none of the block-orthogonalization or GMRES arithmetic; neither the
oracle nor the CUDA library is imported here.

Workload recipes (the paper's experiments use synthetic matrices of these kinds):

* ``glued_blocks``: the "glued" construction of the one-/two-stage experiments
  (Section 8): each block of ``s`` columns is ``U_j diag(sigma) W_j^T`` with
  ``U_j`` the orthonormal factor of a seeded Gaussian n x s matrix, ``W_j`` a
  random s x s orthogonal matrix and ``sigma`` log-spaced from 1 to 1/kappa.
  Optionally a leading Gaussian column ``v0`` is prepended (the V_0 block of
  the paper's notation, Table 1).
* ``poisson3d_csr`` / ``laplace2d_csr``: 7-point and 5-point finite-difference
  Laplacians with Dirichlet boundaries (stencils (6,-1) and (4,-1), unscaled);
  the 2D one is the matrix of the MPK experiment (Section 8, Figure 6), the 3D
  one the matrix of the strong-scaling table (Section 10).
* ``ones_rhs``: b = A * 1, so that the exact solution is the all-ones vector.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "glued_blocks",
    "poisson3d_csr",
    "laplace2d_csr",
    "random_csr",
    "ones_rhs",
    "gaussian_vector",
    "glued_blocks_torch",
    "CSR",
]


def _orthonormal_columns(g: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the columns of a Gaussian matrix (input construction)."""
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def glued_blocks(n: int, nblocks: int, s: int, kappa: float, seed: int = 0,
                 v0: bool = False) -> np.ndarray:
    """Return V (n x (v0 + nblocks*s), float64, column-major) with kappa(V_j) = kappa.

    Each block is U_j diag(logspace(0, -log10(kappa), s)) W_j^T.
    """
    rng = np.random.default_rng(seed)
    ncols = nblocks * s + (1 if v0 else 0)
    V = np.empty((n, ncols), dtype=np.float64, order="F")
    c = 0
    if v0:
        V[:, 0] = rng.standard_normal(n)
        c = 1
    sig = np.logspace(0.0, -np.log10(kappa), s) if s > 1 else np.ones(1)
    for _ in range(nblocks):
        U = _orthonormal_columns(rng.standard_normal((n, s)))
        W = _orthonormal_columns(rng.standard_normal((s, s)))
        V[:, c:c + s] = (U * sig) @ W.T
        c += s
    return V


def gaussian_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)


class CSR:
    """A CSR matrix: int32 row pointers and column indices, float64 values."""

    def __init__(self, n: int, rowptr: np.ndarray, col: np.ndarray, val: np.ndarray):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    @staticmethod
    def from_scipy(a) -> "CSR":
        a = a.tocsr()
        a.sort_indices()
        return CSR(a.shape[0], a.indptr, a.indices, a.data)


def _lap1d(N: int):
    import scipy.sparse as sp
    e = np.ones(N)
    return sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1], format="csr")


def poisson3d_csr(N: int) -> CSR:
    """7-point Laplacian (6 on the diagonal, -1 off) on an N^3 interior grid."""
    import scipy.sparse as sp
    T = _lap1d(N)
    I = sp.identity(N, format="csr")
    A = sp.kron(sp.kron(T, I), I) + sp.kron(sp.kron(I, T), I) + sp.kron(sp.kron(I, I), T)
    return CSR.from_scipy(A)


def laplace2d_csr(N: int) -> CSR:
    """5-point Laplacian (4 on the diagonal, -1 off) on an N^2 interior grid."""
    import scipy.sparse as sp
    T = _lap1d(N)
    I = sp.identity(N, format="csr")
    A = sp.kron(T, I) + sp.kron(I, T)
    return CSR.from_scipy(A)


def random_csr(n: int, per_row: int, seed: int, diag_shift: float = 4.0,
               symmetric: bool = False) -> CSR:
    """Random nonsymmetric sparse matrix with a dominant positive diagonal."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(n), per_row)
    cols = rng.integers(0, n, size=n * per_row)
    vals = rng.standard_normal(n * per_row)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    if symmetric:
        A = A + A.T
    A = A + sp.identity(n) * (diag_shift + np.abs(A).sum(axis=1).A.ravel().mean())
    return CSR.from_scipy(A)


def ones_rhs(A: CSR) -> np.ndarray:
    """b = A * 1 (row sums), whose exact solution is the all-ones vector."""
    rs = np.add.reduceat(A.val, A.rowptr[:-1].astype(np.int64)) if A.nnz else np.zeros(A.n)
    empty = A.rowptr[1:] == A.rowptr[:-1]
    rs[empty] = 0.0
    return rs


def glued_blocks_torch(n: int, nblocks: int, s: int, kappa: float, seed: int,
                       v0: bool, device):
    """GPU-side version of ``glued_blocks`` for sizes too large to build on the host.

    Same recipe (Gaussian -> orthonormal U_j, random orthogonal W_j, log-spaced
    singular values) drawn from torch's generator; values differ from the numpy
    version, the distribution and per-block condition number do not.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    ncols = nblocks * s + (1 if v0 else 0)
    V = torch.empty((ncols, n), dtype=torch.float64, device=device)  # row j = column j
    c = 0
    if v0:
        V[0] = torch.randn(n, generator=g, device=device, dtype=torch.float64)
        c = 1
    sig = torch.logspace(0.0, -float(np.log10(kappa)), s, dtype=torch.float64, device=device)
    for _ in range(nblocks):
        G = torch.randn((n, s), generator=g, device=device, dtype=torch.float64)
        U, Ru = torch.linalg.qr(G)
        U = U * torch.sign(torch.diagonal(Ru))
        Wg = torch.randn((s, s), generator=g, device=device, dtype=torch.float64)
        W, Rw = torch.linalg.qr(Wg)
        W = W * torch.sign(torch.diagonal(Rw))
        V[c:c + s] = ((U * sig) @ W.T).T
        c += s
        del G, U
    return V  # (ncols, n) row-major == n x ncols column-major with ld = n

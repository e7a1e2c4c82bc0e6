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


# ---- convection-diffusion families (learned-preconditioner and stress workloads) ----------
def _smooth_gaussian_field(shape, corr: float, rng) -> np.ndarray:
    """Unit-variance Gaussian random field with covariance ~ exp(-r^2 / (2 corr^2)):
    white noise filtered (periodically) by a Gaussian of standard deviation
    corr / sqrt(2) cells, then renormalised."""
    from scipy import ndimage
    g = rng.standard_normal(shape)
    f = ndimage.gaussian_filter(g, sigma=corr / np.sqrt(2.0), mode="wrap")
    return (f - f.mean()) / f.std()


def convdiff2d_csr(N: int, seed: int, sigma: float = 1.0, corr: float = 32.0,
                   pe_range=(10.0, 1000.0)):
    """2D convection-diffusion -div(k grad u) + w . grad u on the unit square, N x N
    interior cells, Dirichlet boundary, 5-point stencil: diffusion with harmonic-mean
    face diffusivities, first-order upwind convection.  k = exp(sigma g) with g a
    unit-variance Gaussian field of correlation length `corr` cells; w constant with
    a random angle and Peclet number |w| L / mean(k) uniform in `pe_range` (L = 1).
    Returns (CSR, meta)."""
    rng = np.random.default_rng(seed)
    k = np.exp(sigma * _smooth_gaussian_field((N, N), corr, rng))   # k[y, x]
    theta = rng.uniform(0.0, 2.0 * np.pi)
    pe = rng.uniform(*pe_range)
    wmag = pe * k.mean()
    wx, wy = wmag * np.cos(theta), wmag * np.sin(theta)
    h = 1.0 / (N + 1)
    idx = np.arange(N * N).reshape(N, N)
    rows, cols, vals = [], [], []
    diag = np.zeros((N, N))

    def face(a, b):
        return 2.0 * a * b / (a + b)

    # x-direction faces (between (y, x) and (y, x+1)), y-direction faces
    for axis, wcomp in ((1, wx), (0, wy)):
        kn = np.roll(k, -1, axis=axis)
        kp = np.roll(k, 1, axis=axis)
        fplus = face(k, kn)   # face to the +1 neighbour
        fminus = face(k, kp)  # face to the -1 neighbour
        last = [slice(None)] * 2
        first = [slice(None)] * 2
        last[axis] = N - 1
        first[axis] = 0
        fplus[tuple(last)] = k[tuple(last)]     # boundary faces: the cell's own value
        fminus[tuple(first)] = k[tuple(first)]
        diag += (fplus + fminus) / h**2
        conv_p = max(-wcomp, 0.0) / h           # upwind from the + side (w < 0)
        conv_m = max(wcomp, 0.0) / h            # upwind from the - side (w > 0)
        diag += conv_p + conv_m
        # off-diagonals to the +1 neighbour
        sel = [slice(None)] * 2
        sel[axis] = slice(0, N - 1)
        sel = tuple(sel)
        nb = np.roll(idx, -1, axis=axis)
        rows.append(idx[sel].ravel())
        cols.append(nb[sel].ravel())
        vals.append((-fplus[sel] / h**2 - conv_p).ravel())
        sel2 = [slice(None)] * 2
        sel2[axis] = slice(1, N)
        sel2 = tuple(sel2)
        nb2 = np.roll(idx, 1, axis=axis)
        rows.append(idx[sel2].ravel())
        cols.append(nb2[sel2].ravel())
        vals.append((-fminus[sel2] / h**2 - conv_m).ravel())
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    import scipy.sparse as sp
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N * N, N * N))
    return CSR.from_scipy(A), {"peclet": pe, "theta": theta, "wx": wx, "wy": wy, "seed": seed}


def convdiff3d_csr(N: int, seed: int, aniso=(1.0, 1.0, 1e-3), pe: float = 100.0):
    """3D convection-diffusion, 7-point, constant anisotropic diffusion `aniso`,
    first-order upwind convection with a random direction and |w| = pe (L = 1,
    unit mean diffusivity), Dirichlet, N^3 interior cells."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(3)
    w = pe * v / np.linalg.norm(v)
    h = 1.0 / (N + 1)
    import scipy.sparse as sp
    e = np.ones(N)
    I = sp.identity(N, format="csr")
    mats = []
    for ax in range(3):
        T = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1]) * (aniso[ax] / h**2)
        wc = w[ax]
        if wc > 0:
            C = sp.diags([-e[:-1], e], [-1, 0]) * (wc / h)
        else:
            C = sp.diags([e, -e[:-1]], [0, 1]) * (-wc / h)
        D1 = (T + C).tocsr()
        ops = [I, I, I]
        ops[2 - ax] = D1   # x fastest
        mats.append(sp.kron(sp.kron(ops[0], ops[1]), ops[2]))
    A = (mats[0] + mats[1] + mats[2]).tocsr()
    return CSR.from_scipy(A), {"w": w.tolist(), "seed": seed}

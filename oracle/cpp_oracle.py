"""ctypes binding of the C++ oracle (oracle/cpp, test infrastructure only).

The same schemes as the numpy modules of this package, restated in plain C++17 with
loops over column-major float64 arrays (no BLAS): the sparse-sign sketch and its
SplitMix64 draws, the dense kernels (Cholesky with breakdown detection, Householder QR,
triangular solve, long-double Gram), the accuracy measures of equations (1)-(2), the
one-stage and two-stage block orthogonalization schemes, CSR SpMV and s-step GMRES with
the monomial basis, and Householder GMRES (Walker 1988) as the brute-force reference.
Only tests load it; the library never does.  It is built on first use (g++) when the
shared object is missing or older than its sources.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build_cpp

_lib = None

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_I8 = C.POINTER(C.c_int8)
_SIGS = {
    "orc_splitmix64": (C.c_uint64, [C.c_uint64, C.c_uint64]),
    "orc_sparse_sign_entries": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_uint64, _I32, _I8]),
    "orc_sketch_apply": (C.c_int, [C.c_int64, C.c_int32, C.c_int32, C.c_uint64, C.c_int32, _D, _D]),
    "orc_gaussian_entry": (C.c_double, [C.c_uint64, C.c_uint64, C.c_int32, C.c_int32]),
    "orc_cholesky_upper": (C.c_int, [C.c_int32, _D, _D]),
    "orc_householder_qr": (C.c_int, [C.c_int64, C.c_int32, _D, _D, _D]),
    "orc_solve_right_upper": (C.c_int, [C.c_int64, C.c_int32, _D, _D, _D]),
    "orc_gram": (C.c_int, [C.c_int64, C.c_int32, _D, C.c_int32, _D, _D]),
    "orc_orth_error": (C.c_double, [C.c_int64, C.c_int32, _D]),
    "orc_backward_error": (C.c_double, [C.c_int64, C.c_int32, _D, _D, _D]),
    "orc_block_orth": (C.c_int, [C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                 C.c_int32, C.c_int32, C.c_int32, C.c_uint64, _D, _D, _D, _I32]),
    "orc_spmv": (C.c_int, [C.c_int64, _I64, _I32, _D, _D, _D]),
    "orc_sstep_gmres": (C.c_int, [C.c_int64, _I64, _I32, _D, _D, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                  C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, C.c_int32,
                                  C.c_int32, _D, _I32, _D, _D, C.c_int32]),
    "orc_householder_gmres": (C.c_int, [C.c_int64, _I64, _I32, _D, _D, C.c_int32, C.c_double, C.c_int32,
                                        C.c_int32, _D, _I32, _D, _D, C.c_int32]),
}


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_cpp.build())
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _f64(a):
    """Column-major contiguous float64 copy and its pointer."""
    a = np.asfortranarray(np.asarray(a, dtype=np.float64))
    return a, a.ctypes.data_as(_D)


def _out(m, n):
    a = np.zeros((m, n), dtype=np.float64, order="F")
    return a, a.ctypes.data_as(_D)


def _check(code, what):
    if code != 0:
        raise RuntimeError(f"C++ oracle: {what} failed")


def splitmix64(seed: int, i: int) -> int:
    return int(lib().orc_splitmix64(seed, i))


def sparse_sign_entries(row0: int, nrows: int, d: int, zeta: int, seed: int):
    idx = np.zeros((nrows, zeta), dtype=np.int32)
    sgn = np.zeros((nrows, zeta), dtype=np.int8)
    _check(lib().orc_sparse_sign_entries(row0, nrows, d, zeta, seed, idx.ctypes.data_as(_I32),
                                         sgn.ctypes.data_as(_I8)), "sparse_sign_entries")
    return idx, sgn


def sketch_apply(n: int, d: int, zeta: int, seed: int, W) -> np.ndarray:
    W, pw = _f64(W)
    out, po = _out(d, W.shape[1])
    _check(lib().orc_sketch_apply(n, d, zeta, seed, W.shape[1], pw, po), "sketch_apply")
    return np.ascontiguousarray(out)


def gaussian_entry(seed: int, r: int, k: int, d: int) -> float:
    return float(lib().orc_gaussian_entry(seed, r, k, d))


def cholesky_upper(G):
    G, pg = _f64(G)
    R, pr = _out(G.shape[0], G.shape[0])
    info = lib().orc_cholesky_upper(G.shape[0], pg, pr)
    return np.ascontiguousarray(R), int(info)


def householder_qr(A, want_q: bool = False):
    A, pa = _f64(A)
    m, k = A.shape
    R, pr = _out(k, k)
    Q, pq = _out(m, k) if want_q else (None, None)
    _check(lib().orc_householder_qr(m, k, pa, pr, pq), "householder_qr")
    return (np.ascontiguousarray(Q), np.ascontiguousarray(R)) if want_q else np.ascontiguousarray(R)


def solve_right_upper(W, R):
    W, pw = _f64(W)
    R, pr = _f64(R)
    X, px = _out(*W.shape)
    _check(lib().orc_solve_right_upper(W.shape[0], W.shape[1], pw, pr, px), "solve_right_upper")
    return np.ascontiguousarray(X)


def gram(X, Y):
    X, px = _f64(X)
    Y, py = _f64(Y)
    Cm, pc = _out(X.shape[1], Y.shape[1])
    _check(lib().orc_gram(X.shape[0], X.shape[1], px, Y.shape[1], py, pc), "gram")
    return np.ascontiguousarray(Cm)


def orth_error(Q) -> float:
    Q, pq = _f64(Q)
    return float(lib().orc_orth_error(Q.shape[0], Q.shape[1], pq))


def backward_error(V, Q, R) -> float:
    V, pv = _f64(V)
    Q, pq = _f64(Q)
    R, pr = _f64(R)
    return float(lib().orc_backward_error(V.shape[0], V.shape[1], pv, pq, pr))


@dataclass
class OrthResult:
    Q: np.ndarray
    R: np.ndarray
    ok: bool
    breakdown_block: int
    breakdown_column: int


def _orth(scheme, V, s, s_hat, intra, pip, v0, d, zeta, seed):
    V, pv = _f64(V)
    n, c = V.shape
    Q, pq = _out(n, c)
    R, pr = _out(c, c)
    info = np.zeros(3, dtype=np.int32)
    _check(lib().orc_block_orth(scheme, n, c, s, s_hat, intra, pip, int(v0), d, zeta, seed, pv, pq, pr,
                                info.ctypes.data_as(_I32)), "block_orth")
    return OrthResult(np.ascontiguousarray(Q), np.ascontiguousarray(R), bool(info[0]), int(info[1]), int(info[2]))


def block_orth_one_stage(V, s: int, d: int = 0, zeta: int = 8, seed: int = 42, intra: str = "rand",
                         v0: bool = False) -> OrthResult:
    """One-stage BCGS2 (Section 5), RandCholQR (intra="rand") or CholQR2 first step."""
    return _orth(0, V, s, 0, 0 if intra == "rand" else 1, 0, v0, d, zeta, seed)


def block_orth_two_stage(V, s: int, s_hat: int, d: int = 0, zeta: int = 8, seed: int = 42,
                         v0: bool = False, preproc: str = "rand") -> OrthResult:
    """Two-stage scheme (Sections 6-7), RandBCGS2 (preproc="rand") or BCGS-PIP."""
    return _orth(1, V, s, s_hat, 0, 0 if preproc == "rand" else 1, v0, d, zeta, seed)


def _csr(A):
    import scipy.sparse as sp
    M = A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)
    M = M.tocsr()
    rowptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
    col = np.ascontiguousarray(M.indices, dtype=np.int32)
    val = np.ascontiguousarray(M.data, dtype=np.float64)
    return M.shape[0], rowptr, col, val


def spmv(A, x) -> np.ndarray:
    n, rp, col, val = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(n)
    _check(lib().orc_spmv(n, rp.ctypes.data_as(_I64), col.ctypes.data_as(_I32), val.ctypes.data_as(_D),
                          x.ctypes.data_as(_D), y.ctypes.data_as(_D)), "spmv")
    return y


@dataclass
class GmresResult:
    x: np.ndarray
    converged: bool
    iterations: int
    restarts: int
    relres: float
    breakdown: bool
    history: list = field(default_factory=list)


def _gmres_out(fn, n, *args, hist_cap=4096):
    x = np.zeros(n)
    stats = np.zeros(5, dtype=np.int32)
    rel = C.c_double(0.0)
    hist = np.zeros(2 * hist_cap)
    _check(fn(*args, x.ctypes.data_as(_D), stats.ctypes.data_as(_I32), C.byref(rel), hist.ctypes.data_as(_D),
              hist_cap), "gmres")
    h = [(int(hist[2 * i]), float(hist[2 * i + 1])) for i in range(int(stats[4]))]
    return GmresResult(x, bool(stats[2]), int(stats[0]), int(stats[1]), float(rel.value), bool(stats[3]), h)


def sstep_gmres(A, b, *, s: int, m: int, tol: float, s_hat: int | None = None, scheme: str = "one",
                intra: str = "rand", max_restarts: int = 200, d: int | None = None, zeta: int = 8,
                seed: int = 42, precond: str = "jacobi", preproc: str = "rand") -> GmresResult:
    """s-step GMRES(m) (Section 4), monomial basis, one-stage or two-stage."""
    n, rp, col, val = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    s_hat = (s_hat or m) if scheme == "two" else 0
    d = d or 4 * (m + 1)
    return _gmres_out(lib().orc_sstep_gmres, n, n, rp.ctypes.data_as(_I64), col.ctypes.data_as(_I32),
                      val.ctypes.data_as(_D), b.ctypes.data_as(_D), s, m, tol, 0 if scheme == "one" else 1,
                      s_hat, 0 if intra == "rand" else 1, 0 if preproc == "rand" else 1, d, zeta, seed,
                      max_restarts, 1 if precond == "jacobi" else 0)


def householder_gmres(A, b, *, m: int, tol: float, max_restarts: int = 200,
                      precond: str = "jacobi") -> GmresResult:
    """GMRES(m) with Householder-reflector Arnoldi (Walker 1988)."""
    n, rp, col, val = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return _gmres_out(lib().orc_householder_gmres, n, n, rp.ctypes.data_as(_I64), col.ctypes.data_as(_I32),
                      val.ctypes.data_as(_D), b.ctypes.data_as(_D), m, tol, max_restarts,
                      1 if precond == "jacobi" else 0)

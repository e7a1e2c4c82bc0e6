"""Randomized block orthogonalization for s-step GMRES on GB300 (sm_103a).

Thin Python binding of the C ABI in ``include/rbo.h`` (``librbo.so``): argument
marshalling only, every computation runs in the library's CUDA kernels.  PyTorch
provides device memory and the current stream.  Dense n-row matrices are
column-major float64 CUDA tensors: an n x c tensor with ``stride(0) == 1``
(see :func:`colmajor`).

The library is the reference implementation of the paper's hot path:
``sketch_create`` / ``sketch_apply`` (sparse-sign sketch), ``gram``,
``block_orth_one_stage`` / ``block_orth_two_stage`` / ``block_orth_cholqr2``,
``mpk_csr`` and ``sstep_gmres``.  Importing this package fails loudly if the
compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librbo.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -c 'import __graft_entry__ as g; g.build()' or python paper_2503_16717_gb300/build.py)")

lib = C.CDLL(LIB_PATH)

# ---- status codes and modes (mirror include/rbo.h) ---------------------------------------
OK = 0
ERR_ARG = -1
ERR_CUDA = -2
ERR_CHOL_BREAKDOWN = -3
ERR_NOT_CONVERGED = -4
ERR_TIMEOUT = -5
ERR_SKETCH = -6
ERR_NOMEM = -7
ERR_NO_DEVICE = -8
ERR_LOST_ORTHOGONALITY = -9
PREC_FP64 = 0
PREC_MIXED = 1
PREC_DF64 = 2
PREC_OZAKI = 3   # wide Gram passes as exact digit products on the fp16 tensor cores
INTRA_RANDCHOLQR = 0
INTRA_CHOLQR2 = 1
STAGE_NAMES = {0: "", 1: "v0", 2: "intra", 3: "intra2", 4: "final", 5: "bigpanel", 6: "preproc"}
PREPROC_RAND = 0
PREPROC_PIP = 1
BASIS_MONOMIAL = 0
BASIS_NEWTON = 1
BASIS_CHEBYSHEV = 2
SKETCH_SPARSE_SIGN = 0
SKETCH_GAUSSIAN = 1
SKETCH_COUNT_GAUSS = 2


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("v0", C.c_int32), ("intra", C.c_int32),
                ("max_restarts", C.c_int32), ("precond", C.c_int32), ("preproc", C.c_int32),
                ("basis", C.c_int32), ("reserved", C.c_int32 * 1)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("breakdown_block", C.c_int32),
                ("breakdown_column", C.c_int32), ("breakdown_stage", C.c_int32),
                ("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("kernel_launches", C.c_int32), ("relres", C.c_double), ("est_relres", C.c_double),
                ("time_ms", C.c_double), ("history", C.POINTER(C.c_double)),
                ("history_cap", C.c_int32), ("history_len", C.c_int32),
                ("resid", C.c_void_p), ("resid_ld", C.c_int64), ("resid_cap", C.c_int32),
                ("resid_len", C.c_int32), ("fallbacks", C.c_int32)]


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


_vp, _i32, _i64, _u64, _dp = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p

# name -> (restype, argtypes)
SIGNATURES = {
    "rbo_sketch_create": (C.c_int, [_i64, _i32, _i32, _u64, C.POINTER(_vp)]),
    "rbo_sketch_create_ex": (C.c_int, [_i64, _i32, _i32, _i32, _i32, _u64, C.POINTER(_vp)]),
    "rbo_newton_shifts": (C.c_int, [_dp, _i64, _i32, _i32, _dp, _dp]),
    "rbo_chebyshev_shifts": (C.c_int, [_dp, _i64, _i32, _i32, _dp, _dp]),
    "rbo_sketch_destroy": (C.c_int, [_vp]),
    "rbo_sketch_entries": (C.c_int, [_vp, _i64, _i64, _vp, _vp, _vp]),
    "rbo_sketch_apply": (C.c_int, [_vp, _i64, _i32, _vp, _i64, _dp, _i32, _vp]),
    "rbo_gram": (C.c_int, [_i64, _i32, _vp, _i64, _i32, _vp, _i64, _dp, _vp]),
    "rbo_gram_ex": (C.c_int, [_i64, _i32, _vp, _i64, _i32, _vp, _i64, _dp, _i32, _vp]),
    "rbo_gram_noalloc": (C.c_int, [_i64, _i32, _vp, _i64, _i32, _vp, _i64, _vp, _vp]),
    "rbo_block_orth_one_stage": (C.c_int, [_vp, _i64, _i32, _i32, _vp, _i64, _dp, _i64,
                                           C.POINTER(Opts), C.POINTER(Info), _vp]),
    "rbo_block_orth_two_stage": (C.c_int, [_vp, _i64, _i32, _i32, _i32, _vp, _i64, _dp, _i64,
                                           C.POINTER(Opts), C.POINTER(Info), _vp]),
    "rbo_block_orth_cholqr2": (C.c_int, [_i64, _i32, _i32, _vp, _i64, _dp, _i64, C.POINTER(Opts),
                                         C.POINTER(Info), _vp]),
    "rbo_mpk_csr": (C.c_int, [C.POINTER(Csr), _vp, _i32, _vp, _vp, _i64, _vp]),
    "rbo_sstep_gmres": (C.c_int, [C.POINTER(Csr), _vp, _vp, _i32, _i32, _i32, C.c_double, _vp,
                                  C.POINTER(Opts), C.POINTER(Info), _vp]),
    "rbo_sstep_gmres_precond": (C.c_int, [C.POINTER(Csr), _vp, _vp, _vp, _i32, _i32, _i32,
                                          C.c_double, _vp, C.POINTER(Opts), C.POINTER(Info), _vp]),
    "rbo_gnn_param_count": (C.c_int, []),
    "rbo_gnn_create": (C.c_int, [_u64, C.POINTER(_vp)]),
    "rbo_gnn_destroy": (C.c_int, [_vp]),
    "rbo_gnn_set_params": (C.c_int, [_vp, _vp]),
    "rbo_gnn_get_params": (C.c_int, [_vp, _vp]),
    "rbo_gnn_infer": (C.c_int, [_vp, C.POINTER(Csr), _vp, _vp]),
    "rbo_gnn_loss_grad": (C.c_int, [_vp, C.POINTER(Csr), _vp, _i32, _i64, C.POINTER(C.c_double),
                                    _vp, _vp]),
    "rbo_gnn_train_step": (C.c_int, [_vp, C.POINTER(Csr), _vp, _i32, _i64, C.c_float,
                                     C.POINTER(C.c_double), _vp]),
    "rbo_profile_enable": (C.c_int, [C.c_int]),
    "rbo_profile_reset": (C.c_int, []),
    "rbo_profile_read": (C.c_int, [_i32, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "rbo_status_string": (C.c_char_p, [C.c_int]),
    "rbo_release_workspace": (C.c_int, []),
    "rbo_version": (C.c_char_p, []),
    "rbo_last_error": (C.c_char_p, []),
}
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class RboError(RuntimeError):
    def __init__(self, code: int, where: str, info: "Info | None" = None):
        msg = lib.rbo_status_string(code).decode()
        if code == ERR_CUDA:
            msg += " [" + lib.rbo_last_error().decode() + "]"
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code
        self.info = info


def _check(code: int, where: str, info=None):
    if code != OK:
        raise RboError(code, where, info)


# ---- torch plumbing ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _stream():
    return C.c_void_p(_torch().cuda.current_stream().cuda_stream)


def colmajor(n: int, c: int, device="cuda", ld: int | None = None):
    """An n x c float64 CUDA tensor in column-major layout (stride(0) == 1).
    ``ld`` defaults to n rounded up to even (16-byte aligned columns)."""
    torch = _torch()
    ld = ld or (n + (n & 1))
    buf = torch.empty((c, ld), dtype=torch.float64, device=device)
    return buf.t()[:n]


def _mat(V, name: str):
    torch = _torch()
    if not (isinstance(V, torch.Tensor) and V.is_cuda and V.dtype == torch.float64 and V.dim() == 2):
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor")
    if V.shape[1] > 1 and V.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1); use colmajor()")
    ld = V.stride(1) if V.shape[1] > 1 else max(V.shape[0], 1)
    return C.c_void_p(V.data_ptr()), V.shape[0], V.shape[1], ld


def _vec(v, name: str):
    torch = _torch()
    if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64 and v.dim() == 1
            and v.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous 1-D float64 CUDA tensor")
    return C.c_void_p(v.data_ptr())


def info_dict(info: Info) -> dict:
    d = {f: getattr(info, f) for f, _ in Info._fields_ if f not in ("history", "resid")}
    d["breakdown_stage_name"] = STAGE_NAMES.get(info.breakdown_stage, "")
    return d


# ---- sketch ---------------------------------------------------------------------------------
class Sketch:
    """Handle of a sketch S (d x n_max): sparse-sign (zeta entries +-1 per column),
    Gaussian, or Count-Gauss (a d_inner-row Count sketch followed by a Gaussian map)."""

    def __init__(self, n_max: int, d: int, zeta: int = 8, seed: int = 42,
                 kind: int = SKETCH_SPARSE_SIGN, d_inner: int = 0):
        h = C.c_void_p()
        _check(lib.rbo_sketch_create_ex(n_max, d, kind, zeta, d_inner, seed, C.byref(h)),
               "sketch_create")
        self.handle = h
        self.n_max, self.d, self.seed, self.kind, self.d_inner = n_max, d, seed, kind, d_inner
        self.zeta = zeta if kind == SKETCH_SPARSE_SIGN else 1

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.rbo_sketch_destroy(h)
            self.handle = None


def sketch_create(n_max: int, d: int, zeta: int = 8, seed: int = 42,
                  kind: int = SKETCH_SPARSE_SIGN, d_inner: int = 0) -> Sketch:
    return Sketch(n_max, d, zeta, seed, kind, d_inner)


def sketch_entries(sk: Sketch, row0: int, nrows: int):
    """(idx, sign) of sketch columns row0..row0+nrows-1, computed on the GPU."""
    torch = _torch()
    idx = torch.empty((nrows, sk.zeta), dtype=torch.int32, device="cuda")
    sgn = torch.empty((nrows, sk.zeta), dtype=torch.int8, device="cuda")
    _check(lib.rbo_sketch_entries(sk.handle, row0, nrows, C.c_void_p(idx.data_ptr()),
                                  C.c_void_p(sgn.data_ptr()), _stream()), "sketch_entries")
    return idx, sgn


def sketch_apply(sk: Sketch, W, precision: int = PREC_FP64) -> np.ndarray:
    """S W (d x k) for a column-major n x k CUDA tensor W; returned as numpy."""
    p, n, k, ld = _mat(W, "W")
    out = np.zeros((k, sk.d), dtype=np.float64)  # column-major d x k
    _check(lib.rbo_sketch_apply(sk.handle, n, k, p, ld, out.ctypes.data_as(C.c_void_p), precision,
                                _stream()), "sketch_apply")
    return out.T


def gram(X, Y, precision: int = PREC_FP64) -> np.ndarray:
    """X^T Y for column-major CUDA tensors (deterministic tree reduction); precision
    PREC_FP64 or PREC_OZAKI (tensor-core digit products)."""
    px, n, a, ldx = _mat(X, "X")
    py, n2, b, ldy = _mat(Y, "Y")
    if n2 != n:
        raise ValueError("row counts differ")
    out = np.zeros((b, a), dtype=np.float64)
    _check(lib.rbo_gram_ex(n, a, px, ldx, b, py, ldy, out.ctypes.data_as(C.c_void_p), precision,
                           _stream()), "gram")
    return out.T


# ---- block orthogonalization -------------------------------------------------------------------
@dataclass
class OrthOut:
    R: np.ndarray
    info: dict


def _opts(precision=PREC_FP64, v0=False, intra=INTRA_RANDCHOLQR, max_restarts=0, precond=1,
          preproc=PREPROC_RAND, basis=BASIS_MONOMIAL) -> Opts:
    o = Opts()
    o.precision, o.v0, o.intra, o.max_restarts, o.precond = precision, int(v0), intra, max_restarts, precond
    o.preproc, o.basis = preproc, basis
    return o


def _orth_call(fn, args_pre, V, s_args, v0, precision, intra, where, raise_on_error,
               preproc=PREPROC_RAND):
    pv, n, c, ld = _mat(V, "V")
    R = np.zeros((c, c), dtype=np.float64)  # row-major storage of R^T == column-major R
    info = Info()
    o = _opts(precision, v0, intra, preproc=preproc)
    code = fn(*args_pre, n, c, *s_args, pv, ld, R.ctypes.data_as(C.c_void_p), c, C.byref(o),
              C.byref(info), _stream())
    if code != OK and raise_on_error:
        raise RboError(code, where, info)
    return OrthOut(R.T.copy(), info_dict(info))


def block_orth_one_stage(sk: Sketch, V, s: int, v0: bool = False, precision: int = PREC_FP64,
                         intra: int = INTRA_RANDCHOLQR, raise_on_error: bool = True) -> OrthOut:
    """One-stage BCGS2 with RandCholQR (or CholQR2); V (n x c) is overwritten by Q."""
    return _orth_call(lib.rbo_block_orth_one_stage, (sk.handle,), V, (s,), v0, precision, intra,
                      "block_orth_one_stage", raise_on_error)


def block_orth_two_stage(sk: Sketch | None, V, s: int, s_hat: int, v0: bool = False,
                         precision: int = PREC_FP64, raise_on_error: bool = True,
                         preproc: int = PREPROC_RAND) -> OrthOut:
    """Two-stage BCGS2 with RandBCGS2 (or BCGS-PIP: no sketch needed) preprocessing;
    V is overwritten by Q."""
    return _orth_call(lib.rbo_block_orth_two_stage, (sk.handle if sk is not None else None,), V,
                      (s, s_hat), v0, precision, INTRA_RANDCHOLQR, "block_orth_two_stage",
                      raise_on_error, preproc)


def block_orth_cholqr2(V, s: int, v0: bool = False, raise_on_error: bool = True) -> OrthOut:
    """BCGS2 with CholQR2 as the first intra-block step (deterministic baseline)."""
    return _orth_call(lib.rbo_block_orth_cholqr2, (), V, (s,), v0, PREC_FP64, INTRA_CHOLQR2,
                      "block_orth_cholqr2", raise_on_error)


# ---- sparse ------------------------------------------------------------------------------------
class DeviceCSR:
    """A CSR matrix resident on the GPU (int32 rowptr/col, float64 values)."""

    def __init__(self, n: int, rowptr, col, val):
        torch = _torch()
        self.n = int(n)
        self.rowptr = torch.as_tensor(np.asarray(rowptr, dtype=np.int32)).cuda()
        self.col = torch.as_tensor(np.asarray(col, dtype=np.int32)).cuda()
        self.val = torch.as_tensor(np.asarray(val, dtype=np.float64)).cuda()
        self.nnz = int(self.col.numel())

    @staticmethod
    def from_host(A) -> "DeviceCSR":
        return DeviceCSR(A.n, A.rowptr, A.col, A.val)

    def struct(self) -> Csr:
        s = Csr()
        s.n, s.nnz = self.n, self.nnz
        s.rowptr, s.col, s.val = self.rowptr.data_ptr(), self.col.data_ptr(), self.val.data_ptr()
        return s


def mpk_csr(A: DeviceCSR, v0, s: int, V=None, dscale=None):
    """Monomial matrix-powers kernel: V[:, i] = (A D)^{i+1} v0, i < s."""
    if V is None:
        V = colmajor(A.n, s)
    pv, n, c, ld = _mat(V, "V")
    st = A.struct()
    ds = _vec(dscale, "dscale") if dscale is not None else None
    _check(lib.rbo_mpk_csr(C.byref(st), ds, s, _vec(v0, "v0"), pv, ld, _stream()), "mpk_csr")
    return V


def sstep_gmres(A: DeviceCSR, b, x=None, *, s: int = 5, s_hat: int = 0, m: int = 60,
                tol: float = 1e-10, sk: Sketch | None = None, precision: int = PREC_FP64,
                precond: int = 1, max_restarts: int = 0, history_cap: int = 4096,
                M=None, resid=None, intra: int = INTRA_RANDCHOLQR, preproc: int = PREPROC_RAND,
                basis: int = BASIS_MONOMIAL, raise_on_error: bool = False):
    """s-step GMRES(m); returns (x, info).  s_hat in (0, s] -> one-stage, else two-stage.
    ``M``: optional device tensor of preconditioner values on A's pattern (right
    preconditioner; overrides ``precond``)."""
    torch = _torch()
    if x is None:
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    st = A.struct()
    hist = (C.c_double * (2 * history_cap))()
    info = Info()
    info.history = C.cast(hist, C.POINTER(C.c_double))
    info.history_cap = history_cap
    if resid is not None:
        pr, nrr, cap, ldr = _mat(resid, "resid")
        info.resid, info.resid_ld, info.resid_cap = pr.value, ldr, cap
    o = _opts(precision, False, intra, max_restarts, precond, preproc, basis)
    skh = sk.handle if sk is not None else None
    if M is not None:
        code = lib.rbo_sstep_gmres_precond(C.byref(st), _vec(M, "M"), _vec(b, "b"), _vec(x, "x"), s,
                                           s_hat, m, tol, skh, C.byref(o), C.byref(info), _stream())
    else:
        code = lib.rbo_sstep_gmres(C.byref(st), _vec(b, "b"), _vec(x, "x"), s, s_hat, m, tol, skh,
                                   C.byref(o), C.byref(info), _stream())
    d = info_dict(info)
    d["history"] = [(int(hist[2 * i]), float(hist[2 * i + 1])) for i in range(info.history_len)]
    if code != OK and raise_on_error:
        raise RboError(code, "sstep_gmres", info)
    return x, d


def newton_shifts(H, s: int):
    """(alpha, beta) of the Newton basis from the square upper-Hessenberg H (host)."""
    Hf = np.asfortranarray(np.asarray(H, dtype=np.float64))
    k = Hf.shape[0]
    a, b = np.zeros(s), np.zeros(s)
    _check(lib.rbo_newton_shifts(Hf.ctypes.data_as(C.c_void_p), k, k, s, a.ctypes.data_as(C.c_void_p),
                                 b.ctypes.data_as(C.c_void_p)), "newton_shifts")
    return a, b


def chebyshev_shifts(H, s: int):
    """(alpha, beta) of the Chebyshev basis from the square upper-Hessenberg H (host)."""
    Hf = np.asfortranarray(np.asarray(H, dtype=np.float64))
    k = Hf.shape[0]
    a, b = np.zeros(s), np.zeros(s)
    _check(lib.rbo_chebyshev_shifts(Hf.ctypes.data_as(C.c_void_p), k, k, s,
                                    a.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p)),
           "chebyshev_shifts")
    return a, b


# ---- learned SPAI preconditioner -----------------------------------------------------------
GNN_FILE_MAGIC = b"RBOGNN1\0"


def gnn_write(path, theta, seed: int) -> None:
    """Checkpoint of the network's weights: the 8-byte magic, the parameter count
    (uint32) and the creation seed (uint64), little-endian, then the float32 master
    weights in the library's parameter order.  The BF16 copy the kernels use is
    rounded from them when they are loaded."""
    th = np.ascontiguousarray(theta, dtype="<f4").ravel()
    with open(path, "wb") as f:
        f.write(GNN_FILE_MAGIC)
        f.write(np.array([th.size], dtype="<u4").tobytes())
        f.write(np.array([seed], dtype="<u8").tobytes())
        f.write(th.tobytes())


def gnn_read(path):
    """(weights, seed) of a checkpoint written by ``gnn_write``; ValueError for a file
    that is not one or whose parameter count differs from this library's network."""
    with open(path, "rb") as f:
        raw = f.read()
    if len(raw) < 20 or raw[:8] != GNN_FILE_MAGIC:
        raise ValueError(f"{path}: not a network checkpoint")
    count = int(np.frombuffer(raw[8:12], dtype="<u4")[0])
    seed = int(np.frombuffer(raw[12:20], dtype="<u8")[0])
    if count != lib.rbo_gnn_param_count():
        raise ValueError(f"{path}: {count} parameters, the network has {lib.rbo_gnn_param_count()}")
    if len(raw) != 20 + 4 * count:
        raise ValueError(f"{path}: truncated or oversized checkpoint")
    return np.frombuffer(raw[20:], dtype="<f4").astype(np.float32), seed


class GNN:
    """Handle of the learned sparse-approximate-inverse network (BF16 weights, FP32
    master weights and Adam state on the device)."""

    def __init__(self, seed: int = 0):
        h = C.c_void_p()
        _check(lib.rbo_gnn_create(seed, C.byref(h)), "gnn_create")
        self.handle = h
        self.seed = seed
        self.nparam = lib.rbo_gnn_param_count()

    def save(self, path) -> None:
        """Write the weights (not the optimiser state) to a checkpoint file."""
        gnn_write(path, self.get_params(), self.seed)

    @classmethod
    def load(cls, path) -> "GNN":
        """A network with the weights of a checkpoint file."""
        theta, seed = gnn_read(path)
        net = cls(seed)
        net.set_params(theta)
        return net

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.rbo_gnn_destroy(h)
            self.handle = None

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparam, dtype=np.float32)
        _check(lib.rbo_gnn_get_params(self.handle, out.ctypes.data_as(C.c_void_p)), "gnn_get_params")
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        if th.size != self.nparam:
            raise ValueError("wrong parameter count")
        _check(lib.rbo_gnn_set_params(self.handle, th.ctypes.data_as(C.c_void_p)), "gnn_set_params")

    def infer(self, A: "DeviceCSR"):
        torch = _torch()
        M = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
        st = A.struct()
        _check(lib.rbo_gnn_infer(self.handle, C.byref(st), C.c_void_p(M.data_ptr()), _stream()),
               "gnn_infer")
        return M

    def loss_grad(self, A: "DeviceCSR", R):
        pr, n, nr, ldr = _mat(R, "R")
        st = A.struct()
        loss = C.c_double()
        g = np.zeros(self.nparam, dtype=np.float32)
        _check(lib.rbo_gnn_loss_grad(self.handle, C.byref(st), pr, nr, ldr, C.byref(loss),
                                     g.ctypes.data_as(C.c_void_p), _stream()), "gnn_loss_grad")
        return loss.value, g

    def train_step(self, A: "DeviceCSR", R, lr: float = 1e-3) -> float:
        pr, n, nr, ldr = _mat(R, "R")
        st = A.struct()
        loss = C.c_double()
        _check(lib.rbo_gnn_train_step(self.handle, C.byref(st), pr, nr, ldr, lr, C.byref(loss),
                                      _stream()), "gnn_train_step")
        return loss.value


PROF_ROWPASS, PROF_SPMV, PROF_VECTOR, PROF_OZAKI = 0, 1, 2, 3


def profile_enable(on: bool = True):
    lib.rbo_profile_enable(1 if on else 0)


def profile_reset():
    lib.rbo_profile_reset()


def profile_read(kind: int) -> dict:
    """Totals since the last reset for one kernel kind: launches, device ms (CUDA
    events around each launch), algorithmic bytes and flops."""
    n = C.c_int64()
    ms, by, fl = C.c_double(), C.c_double(), C.c_double()
    _check(lib.rbo_profile_read(kind, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)),
           "profile_read")
    return {"launches": n.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}


def release_workspace():
    return lib.rbo_release_workspace()


def version() -> str:
    return lib.rbo_version().decode()

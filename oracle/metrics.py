"""Accuracy measures of a computed QR factorisation (oracle; test infrastructure).

* orthogonality error ||I - Q^T Q||_2          (equation (1), Section 4)
* backward error ||V - Q R||_2 / ||V||_2        (equation (2), Section 4)

Products are formed in numpy's extended ``longdouble`` type so that the
measurement error (about n * 2^-64 on x86, n * 2^-113 on aarch64) stays far
below the 1e-14 level being measured; the resulting small matrices are
rounded to float64 before their 2-norm is taken.
"""
from __future__ import annotations

import numpy as np


def _ld(a):
    return np.asarray(a, dtype=np.longdouble)


def orth_error(Q: np.ndarray) -> float:
    Ql = _ld(Q)
    G = Ql.T @ Ql
    E = (np.eye(Q.shape[1], dtype=np.longdouble) - G).astype(np.float64)
    E = 0.5 * (E + E.T)
    if E.size == 0:
        return 0.0
    return float(np.max(np.abs(np.linalg.eigvalsh(E))))


def backward_error(V: np.ndarray, Q: np.ndarray, R: np.ndarray) -> float:
    D = (_ld(V) - _ld(Q) @ _ld(R)).astype(np.float64)
    nv = np.linalg.norm(np.asarray(V, dtype=np.float64), 2)
    return float(np.linalg.norm(D, 2) / nv) if nv > 0 else float(np.linalg.norm(D, 2))


def rel_diff(A: np.ndarray, B: np.ndarray) -> float:
    """Normwise relative difference ||A - B||_F / ||B||_F."""
    nb = np.linalg.norm(B)
    return float(np.linalg.norm(np.asarray(A) - np.asarray(B)) / (nb if nb > 0 else 1.0))


def cond2(A: np.ndarray) -> float:
    s = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
    return float(s[0] / s[-1]) if s[-1] > 0 else float("inf")

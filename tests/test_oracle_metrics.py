"""Pins of the oracle's accuracy measures (Section 4, equations (1)-(2)):
||I - Q^T Q||_2 and ||V - Q R||_2 / ||V||_2 on constructions whose exact values are
known in closed form, so that a dropped term, a missing symmetrisation, a wrong norm
or a transposed product in the measures fails here."""
import numpy as np
import pytest

from oracle import metrics


def _orthonormal(n, k, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return U


def _rotation(k, seed):
    rng = np.random.default_rng(seed)
    W, _ = np.linalg.qr(rng.standard_normal((k, k)))
    return W


@pytest.mark.parametrize("lams", [
    [3e-11, -1e-12, 0.0, 2e-13, 5e-12],          # one dominant positive eigenvalue
    [1e-13, -7e-11, 4e-12, 0.0, 0.0, 1e-14],     # dominant negative eigenvalue
    [0.25, -0.1, 0.05],                           # large: the quadratic term matters
])
def test_orth_error_of_planted_perturbation(lams):
    # Q = U (I + F) with U orthonormal and F = W diag(lam) W^T symmetric gives
    # Q^T Q = (I + F)^2, so I - Q^T Q = -W diag(2 lam + lam^2) W^T and its 2-norm is
    # max |2 lam + lam^2| (a rotated, non-diagonal error matrix).
    lam = np.array(lams)
    k = len(lam)
    U = _orthonormal(3000, k, 11)
    W = _rotation(k, 12)
    F = W @ np.diag(lam) @ W.T
    Q = U @ (np.eye(k) + F)
    expect = float(np.max(np.abs(2 * lam + lam * lam)))
    got = metrics.orth_error(Q)
    # measurement error: a few float64 roundings of Q itself (|Q| <= 1 + |lam|)
    assert abs(got - expect) <= 1e-15 + 1e-12 * expect, (got, expect)


def test_orth_error_sees_only_column_inner_products():
    # a row permutation and a sign flip of columns leave Q^T Q, hence the measure,
    # unchanged; a wrong product (Q Q^T, n x n) would not be
    U = _orthonormal(500, 4, 13)
    Q = U @ (np.eye(4) + np.diag([1e-10, 0, 0, 0]))
    base = metrics.orth_error(Q)
    perm = np.random.default_rng(14).permutation(500)
    assert abs(metrics.orth_error(Q[perm] * np.array([1, -1, 1, -1])) - base) <= 1e-16
    assert abs(base - (2e-10 + 1e-20)) <= 1e-15


def test_orth_error_of_exact_orthonormal_columns():
    Q = np.zeros((64, 8))
    Q[np.arange(8) * 8, np.arange(8)] = 1.0       # unit vectors: Q^T Q = I exactly
    assert metrics.orth_error(Q) == 0.0
    Q[0, 0] = 2.0                                 # one column of norm 2: error 3
    assert metrics.orth_error(Q) == 3.0


@pytest.mark.parametrize("c,sigma", [(1.0, 1e-14), (3.0, 2e-9), (0.5, 0.5)])
def test_backward_error_of_planted_rank_one_residual(c, sigma):
    # V = Q R + sigma u e_1^T with Q orthonormal (n x k), R = c I and u a unit vector
    # orthogonal to range(Q):  V = [Q u] [c I; sigma e_1^T], so ||V - QR||_2 = sigma and
    # ||V||_2 = sqrt(c^2 + sigma^2) (the first column of the small factor has norm
    # sqrt(c^2 + sigma^2), the others c, and they are orthogonal).
    n, k = 2000, 6
    B = _orthonormal(n, k + 1, 21)
    Q, u = B[:, :k], B[:, k]
    R = c * np.eye(k)
    V = Q @ R
    V[:, 0] += sigma * u
    expect = sigma / np.hypot(c, sigma)
    got = metrics.backward_error(V, Q, R)
    assert abs(got - expect) <= 1e-15 * c / np.hypot(c, sigma) + 1e-12 * expect, (got, expect)


def test_backward_error_uses_spectral_norms():
    # two residual columns of norms 3e-12 and 4e-12 along orthogonal directions:
    # the spectral norm is 4e-12 (a Frobenius norm would give 5e-12)
    n, k = 1000, 3
    B = _orthonormal(n, k + 2, 31)
    Q = B[:, :k]
    R = np.triu(np.ones((k, k)))          # ||Q R||_2 = ||R||_2
    V = Q @ R
    V[:, 0] += 3e-12 * B[:, k]
    V[:, 2] += 4e-12 * B[:, k + 1]
    # ||V||_2: V = [Q B_k B_k+1] [R; 3e-12 e_1^T; 4e-12 e_3^T]; the perturbation moves
    # ||R||_2 by far less than the tolerance below
    nr = np.linalg.norm(R, 2)
    got = metrics.backward_error(V, Q, R)
    assert abs(got - 4e-12 / nr) <= 1e-3 * 4e-12 / nr


def test_rel_diff_is_frobenius_relative():
    A = np.array([[3.0, 0.0], [0.0, 4.0]])
    B = np.array([[3.0, 0.0], [0.0, 0.0]])
    assert metrics.rel_diff(A, B) == 4.0 / 3.0
    assert metrics.rel_diff(B, B) == 0.0

"""Pins of the C++ oracle (oracle/cpp, bound by oracle/cpp_oracle.py) against what the
paper and the mathematics fix, and cross-checks with the numpy oracle.

* SplitMix64 against the published output vectors (tests/golden/splitmix64.txt);
* sparse-sign entries: distinct indices in range, signs +-1, equal to the numpy
  oracle's draws, the sketch apply equal to the dense S W built from those entries;
* Cholesky and Householder QR against planted factors, the breakdown column of a
  singular Gram; the long-double Gram against exact rational arithmetic;
* the accuracy measures (equations (1)-(2)) against planted errors of known 2-norm;
* the schemes: ||I - Q^T Q|| = O(eps) and ||V - QR|| / ||V|| = O(eps) for full-rank
  blocks, R equal to the unique Householder R (non-negative diagonal) within kappa eps,
  CholQR2 breaking down once kappa exceeds eps^(-1/2) while the randomized schemes do
  not (Sections 5.1-5.2);
* s-step GMRES against Householder GMRES (Walker 1988) on small problems: the same
  iteration count within one panel, the solution of A x = A 1.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import cpp_oracle as co
from oracle import krylov, orth
from oracle.sketch import Sketch, gaussian_entries, sparse_sign_entries

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden():
    seeds, cur = {}, None
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("seed"):
            cur = int(line.split()[1])
            seeds[cur] = []
        else:
            seeds[cur].append(int(line))
    return seeds


def test_splitmix64_published_vectors():
    for seed, outs in _golden().items():
        for i, v in enumerate(outs, start=1):
            assert co.splitmix64(seed, i) == v


@pytest.mark.parametrize("row0,d,zeta", [(0, 244, 8), ((1 << 24) - 40, 244, 8), (17, 64, 32), (5, 9, 1)])
def test_sparse_sign_entries(row0, d, zeta):
    idx, sgn = co.sparse_sign_entries(row0, 40, d, zeta, 42)
    assert ((idx >= 0) & (idx < d)).all() and set(np.unique(sgn)) <= {-1, 1}
    for r in range(40):
        assert len(set(idx[r])) == zeta
    i2, s2 = sparse_sign_entries(row0, 40, d, zeta, 42)
    assert np.array_equal(idx, i2) and np.array_equal(sgn, s2)


def test_sketch_apply_is_the_dense_map():
    n, d, zeta = 500, 40, 4
    idx, sgn = co.sparse_sign_entries(0, n, d, zeta, 7)
    S = np.zeros((d, n))
    for r in range(n):
        for t in range(zeta):
            S[idx[r, t], r] += sgn[r, t]
    W = np.random.default_rng(1).standard_normal((n, 3))
    assert np.allclose(co.sketch_apply(n, d, zeta, 7, W), S @ W, rtol=0, atol=1e-13)


def test_gaussian_entries_match_the_numpy_oracle():
    ref = gaussian_entries(42, np.arange(5), 13)
    for r in range(5):
        for k in range(13):
            assert co.gaussian_entry(42, r, k, 13) == ref[r, k]


def test_cholesky_recovers_a_planted_factor_and_reports_breakdown():
    rng = np.random.default_rng(3)
    R0 = np.triu(rng.standard_normal((6, 6))) + 4 * np.eye(6)
    R0[np.diag_indices(6)] = np.abs(R0[np.diag_indices(6)])
    R, info = co.cholesky_upper(R0.T @ R0)
    assert info == -1 and np.allclose(R, R0, rtol=1e-13, atol=1e-13)
    B = rng.standard_normal((10, 4))
    B[:, 2] = B[:, 0] + B[:, 1]           # rank 3: the pivot of column 2 is zero
    G = B.T @ B
    G[2, 2] = (B[:, 0] + B[:, 1]) @ (B[:, 0] + B[:, 1]) - 1e-3   # push it below zero
    assert co.cholesky_upper(G)[1] == 2


def test_householder_qr_recovers_a_planted_factorisation():
    rng = np.random.default_rng(4)
    Q0 = np.linalg.qr(rng.standard_normal((50, 6)))[0]
    R0 = np.triu(rng.standard_normal((6, 6)))
    R0[np.diag_indices(6)] = np.abs(R0[np.diag_indices(6)]) + 1.0
    Q, R = co.householder_qr(Q0 @ R0, want_q=True)
    assert np.allclose(R, R0, atol=1e-12) and np.allclose(Q, Q0, atol=1e-12)
    assert (np.diag(R) >= 0).all() and np.abs(Q.T @ Q - np.eye(6)).max() < 1e-14
    X = co.solve_right_upper(Q0 @ R0, R0)
    assert np.allclose(X, Q0, atol=1e-13)


def test_gram_is_exact_on_small_integers():
    rng = np.random.default_rng(5)
    X = rng.integers(-1000, 1000, (300, 3)).astype(float) / 7.0
    Y = rng.integers(-1000, 1000, (300, 2)).astype(float) / 3.0
    C = co.gram(X, Y)
    for i in range(3):
        for j in range(2):
            exact = sum(Fraction(X[r, i]) * Fraction(Y[r, j]) for r in range(300))
            assert C[i, j] == float(exact)


def test_accuracy_measures_on_planted_errors():
    rng = np.random.default_rng(6)
    U = np.linalg.qr(rng.standard_normal((200, 5)))[0]
    delta = np.array([1e-9, -3e-9, 2e-10, 0.0, 5e-9])
    # Q^T Q = diag((1 + delta)^2): ||I - Q^T Q||_2 = max |(1 + delta_i)^2 - 1|
    assert co.orth_error(U * (1 + delta)) == pytest.approx(np.max(np.abs((1 + delta) ** 2 - 1)), rel=1e-6)
    # V = Q R + t u w^T with unit u, w: ||V - QR||_2 = t
    R = np.triu(rng.standard_normal((5, 5))) + 3 * np.eye(5)
    u = rng.standard_normal(200); u /= np.linalg.norm(u)
    w = rng.standard_normal(5); w /= np.linalg.norm(w)
    V = U @ R + 1e-7 * np.outer(u, w)
    assert co.backward_error(V, U, R) == pytest.approx(1e-7 / np.linalg.norm(V, 2), rel=1e-6)


@pytest.mark.parametrize("scheme", ["one", "two", "two_pip"])
def test_schemes_orthogonalize_full_rank_blocks(scheme):
    V = synth.glued_blocks(3000, 6, 5, 1e4, seed=8, v0=True)
    d = 4 * 31
    if scheme == "one":
        r = co.block_orth_one_stage(V, 5, d=d, v0=True)
    else:
        r = co.block_orth_two_stage(V, 5, 10, d=d, v0=True, preproc="rand" if scheme == "two" else "pip")
    assert r.ok
    assert co.orth_error(r.Q) <= 1e-13
    assert co.backward_error(V, r.Q, r.R) <= 1e-14
    # the QR factorisation with a non-negative diagonal is unique: R agrees with
    # Householder QR of all of V to within kappa(V) eps
    _, Rh = co.householder_qr(V, want_q=True)
    assert np.linalg.norm(r.R - Rh) / np.linalg.norm(Rh) <= 1e-10
    assert np.allclose(np.tril(r.R, -1), 0.0) and (np.diag(r.R) > 0).all()


@pytest.mark.parametrize("scheme", ["one", "two"])
def test_schemes_agree_with_the_numpy_oracle(scheme):
    V = synth.glued_blocks(2000, 6, 5, 1e4, seed=9, v0=True)
    d = 4 * 31
    sk = Sketch(2000, d, 8, 42)
    if scheme == "one":
        r, ref = co.block_orth_one_stage(V, 5, d=d, v0=True), orth.block_orth_one_stage(V, 5, sk, v0=True)
    else:
        r, ref = co.block_orth_two_stage(V, 5, 10, d=d, v0=True), orth.block_orth_two_stage(V, 5, 10, sk, v0=True)
    assert np.linalg.norm(r.R - ref.R) / np.linalg.norm(ref.R) <= 1e-12
    assert np.abs(r.Q - ref.Q).max() <= 1e-10


def test_cholqr2_breaks_down_where_randomized_schemes_do_not():
    # Section 5.1: CholQR squares the condition number, so a block with kappa above
    # eps^(-1/2) ~ 6.7e7 meets a non-positive pivot; RandCholQR (Section 5.2) first
    # preconditions the block with the sketch's R and succeeds
    V = synth.glued_blocks(3000, 4, 5, 1e10, seed=10)
    base = co.block_orth_one_stage(V, 5, intra="cholqr2")
    assert not base.ok and base.breakdown_block >= 0
    r = co.block_orth_one_stage(V, 5, d=4 * 21)
    assert r.ok and co.orth_error(r.Q) <= 1e-13 and co.backward_error(V, r.Q, r.R) <= 1e-14
    t = co.block_orth_two_stage(V, 5, 10, d=4 * 21)
    assert t.ok and co.orth_error(t.Q) <= 1e-13


def test_spmv_matches_scipy():
    A = synth.poisson3d_csr(7)
    x = np.random.default_rng(11).standard_normal(A.n)
    assert np.allclose(co.spmv(A, x), A.to_scipy() @ x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("scheme,s_hat", [("one", None), ("two", 10)])
def test_sstep_gmres_matches_householder_gmres(scheme, s_hat):
    A = synth.poisson3d_csr(8)
    b = synth.ones_rhs(A)
    g = co.sstep_gmres(A, b, s=5, m=30, tol=1e-10, scheme=scheme, s_hat=s_hat)
    h = co.householder_gmres(A, b, m=30, tol=1e-10)
    assert g.converged and h.converged and not g.breakdown
    assert abs(g.iterations - h.iterations) <= (s_hat or 5)
    assert np.abs(g.x - 1.0).max() <= 1e-8 and np.abs(h.x - 1.0).max() <= 1e-8
    # and the numpy oracle's s-step GMRES takes the same iterations
    ref = krylov.sstep_gmres(A, b, s=5, m=30, tol=1e-10, scheme=scheme, s_hat=s_hat)
    assert g.iterations == ref.iterations


def test_householder_gmres_on_a_nonsymmetric_operator_without_preconditioner():
    import scipy.sparse as sp
    rng = np.random.default_rng(12)
    n = 60
    M = sp.diags([4.0 * np.ones(n), -1.3 * np.ones(n - 1), -0.6 * np.ones(n - 1)], [0, -1, 1]).tocsr()
    xs = rng.standard_normal(n)
    h = co.householder_gmres(M, M @ xs, m=20, tol=1e-12, precond="none")
    assert h.converged and np.abs(h.x - xs).max() <= 1e-9

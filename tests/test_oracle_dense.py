"""Pins of the oracle's small dense kernels against library routines and constructions."""
import numpy as np

from oracle.dense import cholesky_upper, gram, householder_qr, solve_right_upper


def test_cholesky_matches_library():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 12))
    G = A.T @ A
    R, info = cholesky_upper(G)
    assert info == -1
    L = np.linalg.cholesky(G)
    assert np.allclose(R, L.T, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.triu(R), R)


def test_cholesky_reports_first_nonpositive_pivot():
    rng = np.random.default_rng(2)
    L = np.tril(rng.standard_normal((6, 6))) + 4 * np.eye(6)
    D = np.diag([1.0, 2.0, 3.0, -1.0, 5.0, 6.0])  # pivot 3 negative
    G = L @ D @ L.T
    R, info = cholesky_upper(G)
    assert info == 3
    G2 = np.diag([1.0, 1.0, 0.0, 1.0])
    assert cholesky_upper(G2)[1] == 2
    G3 = np.eye(3)
    G3[1, 1] = np.nan
    assert cholesky_upper(G3)[1] == 1


def test_householder_matches_library_up_to_signs():
    rng = np.random.default_rng(3)
    for m, k in [(244, 5), (50, 50), (100, 17)]:
        A = rng.standard_normal((m, k))
        Q, R = householder_qr(A, want_q=True)
        Ql, Rl = np.linalg.qr(A)
        s = np.sign(np.diag(Rl))
        assert np.allclose(R, s[:, None] * Rl, atol=1e-12 * np.abs(Rl).max())
        assert np.allclose(Q, Ql * s, atol=1e-12)
        assert (np.diag(R) >= 0).all()
        assert np.allclose(Q.T @ Q, np.eye(k), atol=1e-14 * k)
        assert np.allclose(Q @ R, A, atol=1e-13 * np.abs(A).max())


def test_householder_of_rank_deficient_column():
    A = np.zeros((10, 3))
    A[:, 0] = 1.0
    A[:, 2] = np.arange(10)
    R = householder_qr(A)
    assert abs(R[1, 1]) < 1e-14 and (np.diag(R) >= 0).all()


def test_solve_right_upper():
    rng = np.random.default_rng(4)
    R = np.triu(rng.standard_normal((7, 7))) + 5 * np.eye(7)
    W = rng.standard_normal((30, 7))
    X = solve_right_upper(W, R)
    assert np.allclose(X @ R, W, atol=1e-13)
    assert np.allclose(X, W @ np.linalg.inv(R), atol=1e-12)


def test_gram_exact_on_integer_and_dyadic_data():
    # entries that are small integers times powers of two: every product and partial
    # sum is exact in float64, so C must equal the integer result exactly; columns of
    # very different scales and a cancellation (sum 0) included
    rng = np.random.default_rng(5)
    X = rng.integers(-1000, 1000, size=(3000, 7)).astype(np.float64)
    Y = rng.integers(-1000, 1000, size=(3000, 3)).astype(np.float64)
    X[:, 2] *= 2.0 ** -40
    Y[:, 1] *= 2.0 ** 30
    Xi = X.copy()
    Xi[:, 2] *= 2.0 ** 40
    Yi = Y.copy()
    Yi[:, 1] *= 2.0 ** -30
    exact = (Xi.astype(np.int64).T @ Yi.astype(np.int64)).astype(np.float64)
    exact[2, :] *= 2.0 ** -40
    exact[:, 1] *= 2.0 ** 30
    assert np.array_equal(gram(X, Y), exact)
    Z = np.vstack([X[:10], -X[:10]])
    assert np.array_equal(gram(Z, np.vstack([Y[:10], Y[:10]])), np.zeros((7, 3)))


def test_gram_is_extended_precision():
    # x = (1, 2^-60, -1), y = (1, 1, 1): float64 sums left to right give 0; the
    # extended type (64 significant bits or more) keeps 1 + 2^-60, so the result is
    # the exact 2^-60
    X = np.array([[1.0], [2.0 ** -60], [-1.0]])
    Y = np.ones((3, 1))
    assert gram(X, Y)[0, 0] == 2.0 ** -60

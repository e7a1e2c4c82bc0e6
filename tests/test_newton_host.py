"""The Newton- and Chebyshev-basis recurrences of the library (host code, no GPU
needed) against the oracle's: Ritz values by the library's own Francis QR iteration
versus numpy's eigenvalues, then in modified Leja order (Newton) or through the
smallest-capacity enclosing ellipse (Chebyshev)."""
import numpy as np
import pytest

from oracle import krylov


@pytest.mark.parametrize("k,s", [(2, 2), (3, 3), (10, 5), (30, 10), (61, 5), (128, 20)])
def test_newton_shifts_match_oracle(rbo, k, s):
    rng = np.random.default_rng(k)
    for trial in range(4):
        H = np.triu(rng.standard_normal((k, k)), -1)
        a, b = rbo.newton_shifts(H, s)
        ao, bo = krylov.newton_shifts(H, s)
        scale = max(1.0, np.abs(ao).max(), np.abs(bo).max())
        assert np.abs(a - ao).max() <= 1e-10 * scale
        assert np.abs(b - bo).max() <= 1e-10 * scale


def test_newton_shifts_of_arnoldi_matrix(rbo):
    # an Arnoldi matrix of a nonsymmetric convection-diffusion operator (complex Ritz
    # values), the case the GMRES driver meets
    import synth
    A, _ = synth.convdiff2d_csr(24, seed=5)
    Ahat, _ = krylov.jacobi_scaled(A)
    n, m = Ahat.shape[0], 40
    Q = np.zeros((n, m + 1))
    H = np.zeros((m + 1, m))
    Q[:, 0] = np.random.default_rng(0).standard_normal(n)
    Q[:, 0] /= np.linalg.norm(Q[:, 0])
    for j in range(m):
        w = Ahat @ Q[:, j]
        for i in range(j + 1):
            H[i, j] = Q[:, i] @ w
            w -= H[i, j] * Q[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        Q[:, j + 1] = w / H[j + 1, j]
    a, b = rbo.newton_shifts(H[:m, :m], 10)
    ao, bo = krylov.newton_shifts(H[:m, :m], 10)
    assert np.allclose(a, ao, rtol=1e-10, atol=1e-12) and np.allclose(b, bo, rtol=1e-10, atol=1e-12)
    assert (b >= 0).all()


def test_newton_shifts_bad_arguments(rbo):
    with pytest.raises(rbo.RboError):
        rbo.newton_shifts(np.zeros((0, 0)), 3)


@pytest.mark.parametrize("k,s", [(1, 3), (2, 2), (3, 3), (10, 5), (30, 10), (61, 5), (128, 20)])
def test_chebyshev_shifts_match_oracle(rbo, k, s):
    rng = np.random.default_rng(100 + k)
    for trial in range(4):
        H = np.triu(rng.standard_normal((k, k)), -1)
        a, b = rbo.chebyshev_shifts(H, s)
        ao, bo = krylov.chebyshev_shifts(H, s)
        scale = max(1.0, np.abs(ao).max(), np.abs(bo).max())
        assert np.abs(a - ao).max() <= 1e-9 * scale
        assert np.abs(b - bo).max() <= 1e-9 * scale


def test_chebyshev_shifts_special_cases(rbo):
    # real spectrum: the interval [min, max]; a single pair 2 +- 3i: the segment
    a, b = rbo.chebyshev_shifts(np.diag([0.2, 1.9, 0.7]), 4)
    assert np.allclose(a, 1.05) and np.allclose(b, [0.0, -0.5 * 0.85 ** 2, -0.25 * 0.85 ** 2,
                                                     -0.25 * 0.85 ** 2])
    a, b = rbo.chebyshev_shifts(np.array([[2.0, -3.0], [3.0, 2.0]]), 3)
    assert np.allclose(a, 2.0) and np.allclose(b, [0.0, 4.5, 2.25])
    with pytest.raises(rbo.RboError):
        rbo.chebyshev_shifts(np.zeros((0, 0)), 3)

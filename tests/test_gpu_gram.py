"""GPU parity of the tall-skinny Gram X^T Y (BCGS reduction) against float64 numpy."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,a,b", [(1, 1, 1), (63, 5, 5), (64, 7, 3), (20000, 60, 5),
                                   (100001, 30, 30), (4097, 128, 64), (777, 100, 1)])
def test_gram_matches_numpy(rbo, n, a, b):
    from gpu_util import to_dev
    rng = np.random.default_rng(n + a)
    X = rng.standard_normal((n, a))
    Y = rng.standard_normal((n, b))
    got = rbo.gram(to_dev(X), to_dev(Y))
    ref = (X.astype(np.longdouble).T @ Y.astype(np.longdouble)).astype(np.float64)
    bound = 1e-15 * np.sqrt(n) * (np.abs(X).T @ np.abs(Y)).max() + 1e-300
    assert np.abs(got - ref).max() <= 20 * bound


def test_gram_bitwise_reproducible(rbo):
    from gpu_util import to_dev
    rng = np.random.default_rng(5)
    X = to_dev(rng.standard_normal((1_000_003, 20)))
    Y = to_dev(rng.standard_normal((1_000_003, 5)))
    g1 = rbo.gram(X, Y)
    g2 = rbo.gram(X, Y)
    assert np.array_equal(g1, g2)


def test_gram_unaligned_leading_dimension(rbo):
    import torch
    rng = np.random.default_rng(6)
    n = 5001  # odd ld -> plain-load path instead of bulk copies
    X = rng.standard_normal((n, 9))
    Xd = rbo.colmajor(n, 9, ld=n)
    Xd.copy_(torch.from_numpy(X))
    assert Xd.stride(1) == n
    got = rbo.gram(Xd, Xd)
    assert np.allclose(got, X.T @ X, rtol=1e-12, atol=1e-10)

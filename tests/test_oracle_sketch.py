"""Pins of the oracle's sparse-sign sketch (Section 3 embeddings; SplitMix64 stream)."""
import os

import numpy as np
import pytest

from oracle.sketch import (Sketch, SketchError, candidate_index, draw, sparse_sign_entries,
                           splitmix64_output)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden():
    out = {}
    seed = None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("seed"):
            seed = int(line.split()[1])
            out[seed] = []
        else:
            out[seed].append(int(line))
    return out


def test_splitmix64_published_vectors():
    for seed, vals in _golden().items():
        got = [int(splitmix64_output(seed, i + 1)) for i in range(len(vals))]
        assert got == vals


def test_rows_have_zeta_distinct_indices_in_range():
    idx, sgn = sparse_sign_entries(0, 5000, 244, 8, 42)
    assert idx.shape == (5000, 8) and sgn.shape == (5000, 8)
    assert idx.min() >= 0 and idx.max() < 244
    srt = np.sort(idx, axis=1)
    assert (np.diff(srt, axis=1) > 0).all()
    assert set(np.unique(sgn)) == {-1, 1}


def test_entries_are_a_function_of_the_row_only():
    a_idx, a_sgn = sparse_sign_entries(0, 300, 244, 8, 42)
    b_idx, b_sgn = sparse_sign_entries(100, 150, 244, 8, 42)
    assert np.array_equal(a_idx[100:250], b_idx) and np.array_equal(a_sgn[100:250], b_sgn)


def test_first_entry_is_first_draw():
    # draw 0 of each row is never a duplicate, so it is always entry 0
    idx, sgn = sparse_sign_entries(0, 64, 1000, 4, 7)
    h = draw(7, np.arange(64), 0)
    assert np.array_equal(idx[:, 0], candidate_index(h, 1000))
    assert np.array_equal(sgn[:, 0], np.where(h & np.uint64(1), -1, 1))


def test_index_uniformity_chi_square():
    d = 244
    idx, sgn = sparse_sign_entries(0, 40000, d, 8, 42)
    counts = np.bincount(idx.ravel(), minlength=d)
    expect = idx.size / d
    chi2 = ((counts - expect) ** 2 / expect).sum()
    # d-1 = 243 degrees of freedom: mean 243, sd ~22; 5 sd band
    assert 130 < chi2 < 360
    frac_neg = (sgn < 0).mean()
    assert abs(frac_neg - 0.5) < 0.01


def test_subspace_embedding_distortion():
    # Definition 3.1 / Corollary 3.2 for a scalar multiple of S (the scale is
    # absorbed by the following CholQR): the singular values of c*S*U, U
    # orthonormal, lie in [sqrt(1-mu), sqrt(1+mu)] with the best c giving
    # mu = (smax^2 - smin^2) / (smax^2 + smin^2); a 61-dimensional subspace
    # with d = 4*61 rows must be embedded with mu < 1 (full rank, bounded kappa).
    n, c = 20000, 61
    sk = Sketch(n, 4 * c, 8, 42)
    U, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((n, c)))
    sv = np.linalg.svd(sk.apply(U), compute_uv=False)
    mu = (sv.max() ** 2 - sv.min() ** 2) / (sv.max() ** 2 + sv.min() ** 2)
    assert mu < 0.85
    # a single panel of s+1 = 6 columns is embedded much more tightly
    U6 = U[:, :6]
    sv6 = np.linalg.svd(sk.apply(U6), compute_uv=False)
    assert (sv6.max() ** 2 - sv6.min() ** 2) / (sv6.max() ** 2 + sv6.min() ** 2) < 0.4


def test_apply_matches_definition_on_unit_vectors():
    sk = Sketch(50, 16, 3, 9)
    E = np.eye(50)
    D = sk.apply(E)
    for r in range(50):
        col = np.zeros(16)
        col[sk.idx[r]] = sk.sign[r]
        assert np.array_equal(D[:, r], col)


def test_too_small_d_is_an_error():
    with pytest.raises(SketchError):
        sparse_sign_entries(0, 10, 4, 8, 1)


# --- Gaussian and Count-Gauss maps (Section 5.2) ------------------------------------
def test_gaussian_entries_are_standard_normal():
    from scipy import stats
    from oracle.sketch import gaussian_entries
    g = gaussian_entries(42, np.arange(40000), 25).ravel()
    assert abs(g.mean()) < 5e-3 and abs(g.var() - 1.0) < 1e-2
    assert stats.kstest(g, "norm").pvalue > 1e-3
    # entries are float32 values, a function of (row, sketch row) only
    assert np.array_equal(g.astype(np.float32).astype(np.float64), g)
    sub = gaussian_entries(42, np.array([7, 123]), 25)
    assert np.array_equal(sub, g.reshape(40000, 25)[[7, 123]])
    # neighbouring sketch rows and neighbouring basis rows are uncorrelated draws
    G = g.reshape(40000, 25)
    assert abs(np.corrcoef(G[:, 3], G[:, 4])[0, 1]) < 0.02
    assert abs(np.corrcoef(G[:-1, 0], G[1:, 0])[0, 1]) < 0.02


@pytest.mark.parametrize("kind", ["gauss", "count_gauss"])
def test_gaussian_maps_embed_subspaces(kind):
    # Definition 3.1: a Gaussian map with d = O(k) rows, and the Count-Gauss map with
    # a k^2 Count stage followed by O(k) Gaussian rows, keep a k-dimensional
    # subspace well conditioned (mu < 1); the Gaussian map's mu shrinks as d grows
    from oracle.sketch import CountGaussSketch, GaussianSketch
    n, k = 20000, 10
    U, _ = np.linalg.qr(np.random.default_rng(4).standard_normal((n, k)))
    sk = GaussianSketch(n, 4 * k, 42) if kind == "gauss" else CountGaussSketch(n, 4 * k, k * k, 42)
    sv = np.linalg.svd(sk.apply(U), compute_uv=False)
    mu = (sv.max() ** 2 - sv.min() ** 2) / (sv.max() ** 2 + sv.min() ** 2)
    assert mu < 0.9
    if kind == "gauss":
        sk4 = GaussianSketch(n, 16 * k, 42)
        sv4 = np.linalg.svd(sk4.apply(U), compute_uv=False)
        assert (sv4.max() ** 2 - sv4.min() ** 2) / (sv4.max() ** 2 + sv4.min() ** 2) < mu


def test_count_gauss_is_gaussian_times_count():
    # the Count stage is the zeta = 1 sparse-sign map with the same seed, the
    # Gaussian stage the Gaussian entries over the inner rows
    from oracle.sketch import CountGaussSketch, Sketch, gaussian_entries
    n = 3000
    cg = CountGaussSketch(n, 12, 40, 9)
    C = Sketch(n, 40, 1, 9)
    assert np.array_equal(cg.C.idx, C.idx) and np.array_equal(cg.C.sign, C.sign)
    assert (np.abs(C.dense()).sum(axis=0) == 1).all()        # one +-1 per column
    G = gaussian_entries(9, np.arange(40), 12).T
    W = np.random.default_rng(1).standard_normal((n, 3))
    assert np.allclose(cg.apply(W), G @ (C.dense() @ W), rtol=1e-13, atol=1e-12)

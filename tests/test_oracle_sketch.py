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

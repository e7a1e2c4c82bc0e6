"""GPU parity of the sparse-sign sketch: indices and signs bit-exact against the
oracle, S W within rounding (float64) or float32 error (mixed)."""
import numpy as np
import pytest

import synth
from oracle.sketch import Sketch as OSketch, sparse_sign_entries

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("row0,nrows,d,zeta,seed", [
    (0, 5000, 244, 8, 42),
    (16_777_216 - 3000, 3000, 244, 8, 42),   # last rows of the 2^24-row workload
    (123_456, 777, 404, 8, 7),
    (0, 100, 32, 16, 1),                       # zeta = d/2: many rejected duplicates
    (5, 1000, 2000, 1, 3),                     # Count sketch (zeta = 1)
])
def test_entries_bit_exact(rbo, row0, nrows, d, zeta, seed):
    sk = rbo.sketch_create(row0 + nrows, d, zeta, seed)
    idx, sgn = rbo.sketch_entries(sk, row0, nrows)
    ref_idx, ref_sgn = sparse_sign_entries(row0, nrows, d, zeta, seed)
    assert np.array_equal(idx.cpu().numpy(), ref_idx)
    assert np.array_equal(sgn.cpu().numpy(), ref_sgn)


def test_exhausted_draws_reported_on_both_sides(rbo):
    # zeta == d needs every index of [0, d); 64 draws often do not find all 16, and
    # both implementations must refuse the same way (no silent short column)
    from oracle.sketch import SketchError
    sk = rbo.sketch_create(100, 16, 16, 1)
    with pytest.raises(rbo.RboError) as e:
        rbo.sketch_entries(sk, 0, 100)
    assert e.value.code == rbo.ERR_SKETCH
    with pytest.raises(SketchError):
        sparse_sign_entries(0, 100, 16, 16, 1)


@pytest.mark.parametrize("n,k", [(20000, 5), (12345, 11), (100, 3), (64, 1), (65, 6)])
def test_apply_fp64(rbo, n, k):
    from gpu_util import to_dev
    W = np.random.default_rng(n).standard_normal((n, k))
    sk = rbo.sketch_create(n, 244, 8, 42)
    got = rbo.sketch_apply(sk, to_dev(W))
    ref = OSketch(n, 244, 8, 42).apply(W)
    scale = np.abs(W).max() * np.sqrt(8 * n / 244.0)
    assert np.abs(got - ref).max() <= 1e-13 * scale


def test_apply_mixed_is_float32_accurate(rbo):
    from gpu_util import to_dev
    n, k = 50000, 5
    W = np.random.default_rng(1).standard_normal((n, k))
    sk = rbo.sketch_create(n, 244, 8, 42)
    got = rbo.sketch_apply(sk, to_dev(W), precision=rbo.PREC_MIXED)
    ref = OSketch(n, 244, 8, 42).apply(W)
    scale = np.sqrt(8 * n / 244.0)
    err = np.abs(got - ref).max() / scale
    assert 1e-9 < err < 1e-5   # float32 accumulation, not float64


def test_apply_is_deterministic(rbo):
    from gpu_util import to_dev
    W = to_dev(np.random.default_rng(2).standard_normal((300000, 5)))
    sk = rbo.sketch_create(300000, 244, 8, 42)
    a = rbo.sketch_apply(sk, W)
    b = rbo.sketch_apply(sk, W)
    assert np.array_equal(a, b)


# --- Gaussian and Count-Gauss maps (Section 5.2) ------------------------------------
def test_gaussian_entries_match_generator(rbo):
    # S applied to the unit vectors e_0..e_{n-1} returns S's columns: the GPU's
    # float32 Box-Muller values agree with the oracle's float32-rounded float64
    # evaluation of the same SplitMix64 draws to a few float32 ulps
    import torch
    from oracle.sketch import gaussian_entries
    n, d = 64, 40
    sk = rbo.sketch_create(n, d, seed=11, kind=rbo.SKETCH_GAUSSIAN)
    Wd = rbo.colmajor(n, n)
    Wd.copy_(torch.eye(n, dtype=torch.float64))
    got = rbo.sketch_apply(sk, Wd)                       # d x n
    ref = gaussian_entries(11, np.arange(n), d).T
    assert np.abs(got - ref).max() <= 8 * 2.0 ** -23 * np.abs(ref).max()


@pytest.mark.parametrize("kind", ["gauss", "count_gauss"])
@pytest.mark.parametrize("n,k", [(20000, 5), (12345, 11), (65, 3)])
def test_gaussian_maps_apply(rbo, kind, n, k):
    from gpu_util import to_dev
    from oracle.sketch import CountGaussSketch, GaussianSketch
    W = np.random.default_rng(n + k).standard_normal((n, k))
    if kind == "gauss":
        sk = rbo.sketch_create(n, 2 * k + 2, seed=5, kind=rbo.SKETCH_GAUSSIAN)
        ref = GaussianSketch(n, 2 * k + 2, 5).apply(W)
    else:
        sk = rbo.sketch_create(n, 2 * k + 2, seed=5, kind=rbo.SKETCH_COUNT_GAUSS, d_inner=k * k + 4)
        ref = CountGaussSketch(n, 2 * k + 2, k * k + 4, 5).apply(W)
    got = rbo.sketch_apply(sk, to_dev(W))
    # entries of S differ from the oracle's by float32 ulps; sums of n terms
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    if kind == "count_gauss":
        idx, sgn = rbo.sketch_entries(sk, 0, n)
        ref_idx, ref_sgn = sparse_sign_entries(0, n, k * k + 4, 1, 5)
        assert np.array_equal(idx.cpu().numpy(), ref_idx)
        assert np.array_equal(sgn.cpu().numpy(), ref_sgn)


def test_gaussian_sketch_is_rejected_by_entries(rbo):
    sk = rbo.sketch_create(100, 10, seed=1, kind=rbo.SKETCH_GAUSSIAN)
    with pytest.raises(rbo.RboError):
        rbo.sketch_entries(sk, 0, 10)

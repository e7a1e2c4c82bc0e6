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

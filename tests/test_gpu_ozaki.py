"""GPU parity of the tensor-core Gram (precision mode PREC_OZAKI: exact products of 8-bit
digits on the fp16 tensor cores) against the oracle, and of the orthogonalization
schemes and s-step GMRES in that mode against the float64 tolerances.

Error bound of the digit Gram, per row and tile of 128 rows (Mx, My: the largest
magnitudes of the two columns in the tile): a tile shares its column's fixed-point
scale with the other tiles of its accumulation chunk only while its exponent maximum
stays within two of the scale's, so every value is truncated to a multiple of at most
2^-50 Mx, and the dropped digit pairs (levels 8..12) weigh at most 5 * 2^14 * 2^32 / 2^104
< 2^-55 of Mx My, so |C - X^T Y|_ij <= 2^-48 sum_t 128 Mx My over the tiles t, within
the 2^-47 the test allows."""
import numpy as np
import pytest

import synth
from oracle import metrics
from oracle.dense import gram as ogram

from test_gpu_orth import oracle, run

pytestmark = pytest.mark.gpu

TILE = 128


def _dev(rbo, A):
    import torch
    D = rbo.colmajor(*A.shape)
    D.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    return D


def _bound(X, Y):
    n = X.shape[0]
    nt = (n + TILE - 1) // TILE
    pad = nt * TILE - n
    Xa = np.abs(np.vstack([X, np.zeros((pad, X.shape[1]))])).reshape(nt, TILE, -1).max(axis=1)
    Ya = np.abs(np.vstack([Y, np.zeros((pad, Y.shape[1]))])).reshape(nt, TILE, -1).max(axis=1)
    return 2.0 ** -47 * TILE * (Xa.T @ Ya)


def _scaled(rng, n, k, scales):
    A = rng.standard_normal((n, k))
    return A * np.asarray(scales)[None, :k]


@pytest.mark.parametrize("n,a,b", [(20000, 30, 5), (12347, 59, 5), (1001, 1, 1), (20000, 7, 8),
                                   (128, 56, 8), (333, 63, 1), (100000, 40, 3)])
def test_ozaki_gram_elementwise(rbo, n, a, b):
    rng = np.random.default_rng(n + a + b)
    sx = 10.0 ** rng.uniform(-8, 8, a)
    sy = 10.0 ** rng.uniform(-8, 8, b)
    X = _scaled(rng, n, a, sx)
    Y = _scaled(rng, n, b, sy)
    # a column whose magnitude changes by 1e10 across the rows, one with a single entry
    X[: n // 2, 0] *= 1e-10
    if a > 1:
        X[:, 1] = 0.0
        X[n // 3, 1] = 3.0
    C = rbo.gram(_dev(rbo, X), _dev(rbo, Y), precision=rbo.PREC_OZAKI)
    ref = ogram(X, Y)
    err = np.abs(C - ref)
    assert (err <= _bound(X, Y)).all(), float((err / _bound(X, Y)).max())
    # and close to what the float64 kernel achieves
    C64 = rbo.gram(_dev(rbo, X), _dev(rbo, Y))
    nx = np.linalg.norm(X, axis=0)[:, None] * np.linalg.norm(Y, axis=0)[None, :]
    assert (err <= np.maximum(8 * np.abs(C64 - ref), 2e-15 * nx)).all()


def test_ozaki_gram_special_values(rbo):
    n = 5000
    rng = np.random.default_rng(3)
    X = rng.standard_normal((n, 6))
    Y = rng.standard_normal((n, 3))
    X[:, 0] = 0.0                       # a zero column
    X[:, 1] *= 1e-300                   # near the bottom of the float64 range
    X[:, 2] *= 1e300                    # near the top
    Y[:, 2] *= 1e-5
    X[7, 3] = 5e-320                    # a subnormal value (treated as 0 beside normals)
    C = rbo.gram(_dev(rbo, X), _dev(rbo, Y), precision=rbo.PREC_OZAKI)
    ref = ogram(X, Y)
    assert (C[0] == 0.0).all()
    err = np.abs(C - ref)
    assert (err <= _bound(X, Y) + 1e-318).all()
    X[11, 4] = np.nan
    Y[13, 1] = np.inf
    C = rbo.gram(_dev(rbo, X), _dev(rbo, Y), precision=rbo.PREC_OZAKI)
    assert np.isnan(C[4]).all() and np.isnan(C[:, 1]).all()
    ok = np.ones_like(C, dtype=bool)
    ok[4] = False
    ok[:, 1] = False
    assert np.isfinite(C[ok]).all()


def test_ozaki_gram_deterministic_and_rejects_wide_shapes(rbo):
    rng = np.random.default_rng(4)
    X = _dev(rbo, rng.standard_normal((70001, 33)))
    Y = _dev(rbo, rng.standard_normal((70001, 4)))
    C1 = rbo.gram(X, Y, precision=rbo.PREC_OZAKI)
    C2 = rbo.gram(X, Y, precision=rbo.PREC_OZAKI)
    assert np.array_equal(C1, C2)
    with pytest.raises(Exception):
        rbo.gram(_dev(rbo, rng.standard_normal((100, 65))), _dev(rbo, rng.standard_normal((100, 4))),
                 precision=rbo.PREC_OZAKI)
    with pytest.raises(Exception):
        rbo.gram(X, _dev(rbo, rng.standard_normal((70001, 9))), precision=rbo.PREC_OZAKI)


# ---- the schemes in the tensor-core mode meet the float64 tolerances ------------------------
@pytest.mark.parametrize("scheme,s_hat", [("one", None), ("two", 30), ("two", 10)])
@pytest.mark.parametrize("n", [20000, 12347, 1001])
def test_ozaki_orth_well_conditioned_elementwise(rbo, scheme, s_hat, n):
    V = synth.glued_blocks(n, 12, 5, 1e4, seed=n, v0=True)
    Q, out = run(rbo, scheme, V, 5, s_hat, v0=True, precision=rbo.PREC_OZAKI)
    ref = oracle(scheme, V, 5, s_hat, v0=True)
    assert out.info["status"] == 0 and ref.ok
    assert metrics.rel_diff(out.R, ref.R) <= 1e-12
    assert np.abs(Q - ref.Q).max() <= 1e-9
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14
    assert np.allclose(np.tril(out.R, -1), 0.0) and (np.diag(out.R) > 0).all()


@pytest.mark.parametrize("scheme,s_hat", [("one", None), ("two", 30), ("two", 60)])
def test_ozaki_config0_kappa_1e10(rbo, scheme, s_hat):
    V = synth.glued_blocks(20000, 12, 5, 1e10, seed=0)
    Q, out = run(rbo, scheme, V, 5, s_hat, d=244, precision=rbo.PREC_OZAKI)
    assert out.info["status"] == 0
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14
    ref = oracle(scheme, V, 5, s_hat, d=244)
    for j in range(12):
        c_gpu = metrics.cond2(out.R[5 * j:5 * j + 5, 5 * j:5 * j + 5])
        c_ref = metrics.cond2(ref.R[5 * j:5 * j + 5, 5 * j:5 * j + 5])
        assert abs(np.log10(c_gpu) - np.log10(c_ref)) < 0.01
    assert metrics.rel_diff(out.R, ref.R) <= 1e-4


@pytest.mark.parametrize("kappa", [1e4, 1e8, 1e12, 1e14])
@pytest.mark.parametrize("scheme", ["one", "two"])
def test_ozaki_kappa_sweep(rbo, scheme, kappa):
    V = synth.glued_blocks(30000, 12, 5, kappa, seed=17, v0=True)
    Q, out = run(rbo, scheme, V, 5, 30, v0=True, precision=rbo.PREC_OZAKI)
    assert out.info["status"] == 0
    assert metrics.orth_error(Q) <= 1e-13
    assert metrics.backward_error(V, Q, out.R) <= 1e-14


@pytest.mark.parametrize("n,s,nb", [(7, 1, 5), (64, 5, 2), (65, 5, 2), (129, 16, 8), (3, 3, 1)])
def test_ozaki_edge_shapes(rbo, n, s, nb):
    V = synth.glued_blocks(n, nb, s, 10.0, seed=n)
    Q, out = run(rbo, "one", V, s, d=max(4 * (nb * s + 1), 16), precision=rbo.PREC_OZAKI)
    ref = oracle("one", V, s, d=max(4 * (nb * s + 1), 16))
    assert out.info["status"] == 0
    assert metrics.rel_diff(out.R, ref.R) <= 1e-12
    assert metrics.orth_error(Q) <= 1e-13


@pytest.mark.parametrize("s_hat", [0, 10])
def test_ozaki_gmres_matches_oracle(rbo, s_hat):
    import torch
    from oracle import krylov as okry
    A = synth.poisson3d_csr(20)
    b = synth.ones_rhs(A)
    Ad = rbo.DeviceCSR.from_host(A)
    bd = torch.from_numpy(b).cuda()
    x, info = rbo.sstep_gmres(Ad, bd, s=5, s_hat=s_hat, m=30, tol=1e-10, precision=rbo.PREC_OZAKI)
    kw = dict(scheme="two", s_hat=s_hat) if s_hat else {}
    ref = okry.sstep_gmres(A, b, s=5, m=30, tol=1e-10, **kw)
    assert info["status"] == 0 and info["converged"] == 1
    gran = s_hat or 5
    assert abs(info["iterations"] - ref.iterations) <= gran
    assert np.abs(x.cpu().numpy() - 1.0).max() <= 1e-6

"""GPU parity of the matrix-powers kernel and s-step GMRES against the oracle.

GMRES parity: converged to tol on the true residual, iteration count within one
check granularity (s for one-stage, s_hat for two-stage) of the oracle's, and
b = A*1 recovers x = 1."""
import numpy as np
import pytest

import synth
from oracle import krylov

pytestmark = pytest.mark.gpu


def test_mpk_matches_oracle(rbo):
    import torch
    A = synth.poisson3d_csr(20)
    Ad = rbo.DeviceCSR.from_host(A)
    u = np.random.default_rng(0).standard_normal(A.n)
    V = rbo.mpk_csr(Ad, torch.from_numpy(u).cuda(), 5)
    ref = krylov.mpk(A.to_scipy(), u, 5)
    got = V.cpu().numpy()
    for i in range(5):
        assert np.abs(got[:, i] - ref[:, i]).max() <= 1e-13 * np.abs(ref[:, i]).max()


def test_mpk_jacobi_scaled(rbo):
    import torch
    A = synth.random_csr(3001, 9, seed=4)
    Ad = rbo.DeviceCSR.from_host(A)
    u = np.random.default_rng(1).standard_normal(A.n)
    Ahat, dinv = krylov.jacobi_scaled(A)
    V = rbo.mpk_csr(Ad, torch.from_numpy(u).cuda(), 3, dscale=torch.from_numpy(dinv).cuda())
    ref = krylov.mpk(Ahat, u, 3)
    assert np.allclose(V.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _irregular_csr(seed, max_len=9, n=1037):
    """Short rows with empty rows, one row spanning several 256-entry chunks and a
    row count that is not a multiple of 32 (the short-row kernel: about 4.8 entries
    per row at max_len = 9, 8.5 at max_len = 17)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, max_len, size=n)
    lens[rng.choice(n, 40, replace=False)] = 0
    lens[500], lens[31], lens[n - 1] = 700, 300, 12
    rows = np.repeat(np.arange(n), lens)
    cols = np.concatenate([rng.choice(n, k, replace=False) for k in lens])
    A = sp.csr_matrix((rng.standard_normal(rows.size), (rows, cols)), shape=(n, n))
    A.sort_indices()
    return synth.CSR.from_scipy(A)


@pytest.mark.parametrize("max_len,n", [(9, 1037), (17, 1037), (9, 70001), (3, 4099)])
def test_spmv_irregular_rows(rbo, max_len, n):
    import torch
    A = _irregular_csr(3, max_len, n)
    assert 0 < A.nnz / A.n <= 12  # the short-row kernels
    u = np.random.default_rng(2).standard_normal(A.n)
    V = rbo.mpk_csr(rbo.DeviceCSR.from_host(A), torch.from_numpy(u).cuda(), 2)
    ref = krylov.mpk(A.to_scipy(), u, 2)
    got = V.cpu().numpy()
    for i in range(2):
        assert np.abs(got[:, i] - ref[:, i]).max() <= 1e-13 * np.abs(ref[:, i]).max()


@pytest.mark.parametrize("max_len", [9, 17])
@pytest.mark.parametrize("where", ["long", "short"])
def test_spmv_column_out_of_range_is_reported(rbo, max_len, where):
    # a bad index inside the long row (a group of several chunks) and inside a short row
    import torch
    A = _irregular_csr(4, max_len)
    lens = np.diff(A.rowptr)
    row = 500 if where == "long" else next(r for r in range(600, A.n) if 4 <= lens[r] <= 16)
    A.col[A.rowptr[row] + 3] = A.n + 5
    with pytest.raises(rbo.RboError) as e:
        rbo.mpk_csr(rbo.DeviceCSR.from_host(A), torch.ones(A.n, dtype=torch.float64).cuda(), 1)
    assert e.value.code == rbo.ERR_ARG


@pytest.mark.parametrize("N,s,s_hat,m", [(16, 5, 0, 30), (16, 5, 10, 30), (20, 5, 20, 60),
                                         (12, 3, 0, 12), (16, 10, 0, 60), (16, 15, 0, 30),
                                         (16, 10, 30, 60)])
def test_poisson_matches_oracle(rbo, N, s, s_hat, m):
    import torch
    A = synth.poisson3d_csr(N)
    b = synth.ones_rhs(A)
    Ad = rbo.DeviceCSR.from_host(A)
    x, info = rbo.sstep_gmres(Ad, torch.from_numpy(b).cuda(), s=s, s_hat=s_hat, m=m, tol=1e-10)
    scheme = "two" if s_hat > s else "one"
    ref = krylov.sstep_gmres(A, b, s=s, m=m, s_hat=(s_hat or None), scheme=scheme, tol=1e-10)
    assert info["converged"] == 1 and ref.converged
    gran = s_hat if s_hat > s else s
    assert abs(info["iterations"] - ref.iterations) <= gran
    xh = x.cpu().numpy()
    r = b - A.to_scipy() @ xh
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    assert np.abs(xh - 1.0).max() <= 1e-6
    # restart histories agree while rounding has not diverged (with s > 5 the
    # monomial panels are so ill-conditioned that the first cycle's residuals are
    # decided by rounding)
    h = dict(ref.history) if s <= 5 else {}
    for it, rel in info["history"][:3]:
        if it in h and h[it] > 1e-8:
            assert abs(rel - h[it]) <= 1e-6 * h[it]


def test_nonsymmetric_and_resume(rbo):
    import torch
    A = synth.random_csr(5000, 7, seed=11)
    b = np.random.default_rng(3).standard_normal(A.n)
    Ad = rbo.DeviceCSR.from_host(A)
    bd = torch.from_numpy(b).cuda()
    x1, i1 = rbo.sstep_gmres(Ad, bd, s=5, m=20, tol=1e-4)
    assert i1["converged"] == 1
    x2, i2 = rbo.sstep_gmres(Ad, bd, x1.clone(), s=5, m=20, tol=1e-11)
    assert i2["converged"] == 1 and i2["history"][0][1] <= 1e-4
    ref = krylov.sstep_gmres(A, b, s=5, m=20, tol=1e-11)
    xr = x2.cpu().numpy()
    assert np.linalg.norm(b - A.to_scipy() @ xr) / np.linalg.norm(b) <= 1e-11
    assert np.abs(xr - ref.x).max() <= 1e-8 * np.abs(ref.x).max()


def test_not_converged_status(rbo):
    import torch
    A = synth.poisson3d_csr(16)
    b = synth.ones_rhs(A)
    Ad = rbo.DeviceCSR.from_host(A)
    x, info = rbo.sstep_gmres(Ad, torch.from_numpy(b).cuda(), s=5, m=10, tol=1e-12, max_restarts=2)
    assert info["status"] == rbo.ERR_NOT_CONVERGED and info["converged"] == 0
    assert info["restarts"] == 2


def test_zero_rhs(rbo):
    import torch
    A = synth.poisson3d_csr(8)
    Ad = rbo.DeviceCSR.from_host(A)
    x, info = rbo.sstep_gmres(Ad, torch.zeros(A.n, dtype=torch.float64, device="cuda"), s=5, m=10)
    assert info["converged"] == 1 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("s_hat", [0, 20])
def test_poisson_df64_matches_oracle(rbo, s_hat):
    import torch
    A = synth.poisson3d_csr(20)
    b = synth.ones_rhs(A)
    Ad = rbo.DeviceCSR.from_host(A)
    x, info = rbo.sstep_gmres(Ad, torch.from_numpy(b).cuda(), s=5, s_hat=s_hat, m=60, tol=1e-10,
                              precision=rbo.PREC_DF64)
    ref = krylov.sstep_gmres(A, b, s=5, m=60, s_hat=(s_hat or None),
                             scheme="two" if s_hat else "one", tol=1e-10)
    assert info["converged"] == 1
    assert abs(info["iterations"] - ref.iterations) <= (s_hat or 5)
    assert np.abs(x.cpu().numpy() - 1.0).max() <= 1e-6


def test_mixed_precision_falls_back_to_float64_cycle(rbo):
    # s = 10 monomial panels of a 3D convection-diffusion matrix: the float32 sketch
    # cannot precondition some big panel, the cycle is redone in float64 and the
    # solve converges with the float64 solve's iteration count
    import torch
    Ah, _ = synth.convdiff3d_csr(32, seed=7)
    A = rbo.DeviceCSR.from_host(Ah)
    b = torch.from_numpy(synth.ones_rhs(Ah)).cuda()
    _, im = rbo.sstep_gmres(A, b, s=10, s_hat=50, m=100, tol=1e-10, precision=rbo.PREC_MIXED)
    _, i64 = rbo.sstep_gmres(A, b, s=10, s_hat=50, m=100, tol=1e-10)
    assert im["status"] == 0 and im["converged"] == 1 and im["relres"] <= 1e-10
    assert im["fallbacks"] >= 1 and i64["fallbacks"] == 0
    assert abs(im["iterations"] - i64["iterations"]) <= 50


@pytest.mark.parametrize("s", [5, 10])
def test_cholqr2_intra_matches_oracle(rbo, s):
    # the deterministic baseline inside GMRES (opts.intra): same iterations as the
    # oracle's s-step GMRES with CholQR2, or both break down
    import torch
    A = synth.poisson3d_csr(14)
    b = synth.ones_rhs(A)
    Ad = rbo.DeviceCSR.from_host(A)
    x, info = rbo.sstep_gmres(Ad, torch.from_numpy(b).cuda(), s=s, m=30, tol=1e-10,
                              intra=rbo.INTRA_CHOLQR2)
    try:
        ref = krylov.sstep_gmres(A, b, s=s, m=30, scheme="one", intra="cholqr2", tol=1e-10)
        ref_ok = ref.converged
    except Exception:
        ref_ok = False
    if info["status"] == 0:
        assert ref_ok
        assert abs(info["iterations"] - ref.iterations) <= s
    else:
        assert info["status"] in (rbo.ERR_CHOL_BREAKDOWN, rbo.ERR_LOST_ORTHOGONALITY)
    with pytest.raises(rbo.RboError):
        rbo.sstep_gmres(Ad, torch.from_numpy(b).cuda(), s=5, s_hat=10, m=30, tol=1e-10,
                        intra=rbo.INTRA_CHOLQR2, raise_on_error=True)


@pytest.mark.parametrize("N,s_hat", [(16, 10), (20, 10)])
def test_two_stage_pip_gmres_matches_oracle(rbo, N, s_hat):
    # (with s_hat = 20 the monomial big panels reach kappa ~ eps^{-1/2}, where
    # whether the Pythagorean Cholesky breaks down is decided by rounding)
    import torch
    A = synth.poisson3d_csr(N)
    b = synth.ones_rhs(A)
    x, info = rbo.sstep_gmres(rbo.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), s=5,
                              s_hat=s_hat, m=60, tol=1e-10, preproc=rbo.PREPROC_PIP)
    ref = krylov.sstep_gmres(A, b, s=5, m=60, s_hat=s_hat, scheme="two", tol=1e-10, preproc="pip")
    assert info["converged"] == 1 and ref.converged
    assert abs(info["iterations"] - ref.iterations) <= s_hat
    assert np.abs(x.cpu().numpy() - 1.0).max() <= 1e-6


@pytest.mark.parametrize("kind", ["gauss", "count_gauss"])
def test_gmres_with_gaussian_sketches(rbo, kind):
    import torch
    A = synth.poisson3d_csr(16)
    b = synth.ones_rhs(A)
    Ad = rbo.DeviceCSR.from_host(A)
    bd = torch.from_numpy(b).cuda()
    if kind == "gauss":
        sk = rbo.sketch_create(A.n, 2 * 21, seed=42, kind=rbo.SKETCH_GAUSSIAN)
    else:
        sk = rbo.sketch_create(A.n, 2 * 21, seed=42, kind=rbo.SKETCH_COUNT_GAUSS, d_inner=400)
    for s_hat in (5, 20):
        x, info = rbo.sstep_gmres(Ad, bd, s=5, s_hat=s_hat, m=60, tol=1e-10, sk=sk)
        _, ref = rbo.sstep_gmres(Ad, bd, s=5, s_hat=s_hat, m=60, tol=1e-10)
        assert info["converged"] == 1
        assert abs(info["iterations"] - ref["iterations"]) <= s_hat
        assert np.abs(x.cpu().numpy() - 1.0).max() <= 1e-6


@pytest.mark.parametrize("basis", ["newton", "chebyshev"])
@pytest.mark.parametrize("N,s,s_hat,m", [(16, 5, 0, 30), (16, 10, 0, 60), (16, 5, 10, 30),
                                         (16, 30, 0, 60), (16, 20, 60, 60)])
def test_newton_basis_gmres_matches_oracle(rbo, N, s, s_hat, m, basis):
    # the Newton and Chebyshev bases keep large s usable: the first cycle is standard
    # GMRES, later panels of s shifted vectors stay well conditioned (monomial s = 30
    # panels are numerically rank deficient)
    import torch
    A = synth.poisson3d_csr(N)
    b = synth.ones_rhs(A)
    code = rbo.BASIS_NEWTON if basis == "newton" else rbo.BASIS_CHEBYSHEV
    x, info = rbo.sstep_gmres(rbo.DeviceCSR.from_host(A), torch.from_numpy(b).cuda(), s=s,
                              s_hat=s_hat, m=m, tol=1e-10, basis=code)
    scheme = "two" if s_hat > s else "one"
    ref = krylov.sstep_gmres(A, b, s=s, m=m, s_hat=(s_hat or None), scheme=scheme, tol=1e-10,
                             basis=basis)
    assert info["status"] == 0 and info["converged"] == 1 and ref.converged
    gran = s_hat if s_hat > s else s
    assert abs(info["iterations"] - ref.iterations) <= gran
    assert np.abs(x.cpu().numpy() - 1.0).max() <= 1e-6


@pytest.mark.parametrize("basis", ["newton", "chebyshev"])
def test_newton_basis_nonsymmetric(rbo, basis):
    # complex Ritz values: conjugate pairs in the Newton recurrence, an ellipse (not an
    # interval) for the Chebyshev basis
    import torch
    A, _ = synth.convdiff2d_csr(48, seed=1002)
    b = synth.ones_rhs(A)
    Ad = rbo.DeviceCSR.from_host(A)
    bd = torch.from_numpy(b).cuda()
    code = rbo.BASIS_NEWTON if basis == "newton" else rbo.BASIS_CHEBYSHEV
    x, info = rbo.sstep_gmres(Ad, bd, s=10, m=60, tol=1e-10, basis=code)
    ref = krylov.sstep_gmres(A, b, s=10, m=60, tol=1e-10, basis=basis)
    assert info["converged"] == 1 and ref.converged
    assert abs(info["iterations"] - ref.iterations) <= 10
    r = b - A.to_scipy() @ x.cpu().numpy()
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10
    with pytest.raises(rbo.RboError) as e:
        rbo.sstep_gmres(Ad, bd, s=10, m=60, tol=1e-10, basis=3, raise_on_error=True)
    assert e.value.code == rbo.ERR_ARG

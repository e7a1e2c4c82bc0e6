"""Pins of the oracle's MPK and s-step GMRES: GMRES minimises the residual over the
same Krylov space whatever the basis, so at multiples of s the s-step residual
estimates equal those of Householder-Arnoldi GMRES (Walker 1988); b = A*1 gives
x = 1; s_hat = s reduces the two-stage solver to the one-stage one."""
import numpy as np
import pytest

import synth
from oracle import krylov


@pytest.fixture(scope="module")
def small():
    A = synth.random_csr(150, 5, seed=3)
    return A, synth.ones_rhs(A)


def test_spmv_and_mpk_match_dense(small):
    A, _ = small
    D = A.to_scipy().toarray()
    u = np.random.default_rng(0).standard_normal(A.n)
    assert np.allclose(krylov.spmv(A, u), D @ u, atol=1e-13)
    V = krylov.mpk(A.to_scipy(), u, 4)
    assert np.allclose(V[:, 3], np.linalg.matrix_power(D, 4) @ u, rtol=1e-12)


@pytest.mark.parametrize("scheme,s_hat,preproc", [("one", None, "rand"), ("two", 10, "rand"),
                                                  ("two", 20, "rand"), ("two", 10, "pip")])
def test_sstep_estimates_equal_householder_gmres(scheme, s_hat, preproc):
    A = synth.laplace2d_csr(20)
    b = synth.ones_rhs(A)
    ref = dict(krylov.householder_gmres(A, b, m=20, tol=1e-11, max_restarts=2).estimates)
    g = krylov.sstep_gmres(A, b, s=5, m=20, s_hat=s_hat, scheme=scheme, tol=1e-11, max_restarts=2,
                           preproc=preproc)
    checked = 0
    for it, est in g.estimates:
        if it <= 40:
            assert abs(est - ref[it]) <= 1e-9 * ref[it]
            checked += 1
    assert checked >= 2


def test_restarted_histories_agree(small):
    A, b = small
    ref = krylov.householder_gmres(A, b, m=10, tol=1e-10, max_restarts=10)
    g = krylov.sstep_gmres(A, b, s=5, m=10, tol=1e-10, max_restarts=10)
    # full restart cycles end at the same iteration counts with the same residual
    h1 = dict(ref.history)
    common = [(i, r) for i, r in g.history if i in h1 and i % 10 == 0]
    assert len(common) >= 2
    for i, r in common:
        assert abs(r - h1[i]) <= 1e-8 * h1[i]


def test_poisson_solution_is_ones():
    A = synth.poisson3d_csr(16)
    b = synth.ones_rhs(A)
    for scheme, s_hat in [("one", None), ("two", 20)]:
        g = krylov.sstep_gmres(A, b, s=5, m=60, s_hat=s_hat, scheme=scheme, tol=1e-10)
        assert g.converged and g.relres <= 1e-10
        assert np.abs(g.x - 1.0).max() <= 1e-7
        r = b - A.to_scipy() @ g.x
        assert np.linalg.norm(r) / np.linalg.norm(b) <= 1e-10


def test_two_stage_s_hat_equal_s_matches_one_stage():
    A = synth.poisson3d_csr(10)
    b = synth.ones_rhs(A)
    a = krylov.sstep_gmres(A, b, s=5, m=20, tol=1e-10)
    c = krylov.sstep_gmres(A, b, s=5, m=20, s_hat=5, scheme="two", tol=1e-10)
    assert a.iterations == c.iterations
    assert np.allclose(a.x, c.x, atol=1e-9)


def test_x0_resume():
    A = synth.poisson3d_csr(10)
    b = synth.ones_rhs(A)
    g1 = krylov.sstep_gmres(A, b, s=5, m=20, tol=1e-4)
    g2 = krylov.sstep_gmres(A, b, g1.x, s=5, m=20, tol=1e-10)
    assert g2.converged and g2.history[0][1] <= 1e-4 * 1.0001

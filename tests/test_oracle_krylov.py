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


# --- Newton basis (Bai, Hu and Reichel 1994) -----------------------------------------
def test_newton_estimates_equal_householder_gmres():
    # later cycles use the Newton basis of the first cycle's Ritz values; it spans the
    # same Krylov space, so the residual estimates stay those of Householder GMRES
    A = synth.laplace2d_csr(20)
    b = synth.ones_rhs(A)
    ref = dict(krylov.householder_gmres(A, b, m=20, tol=1e-11, max_restarts=3).estimates)
    g = krylov.sstep_gmres(A, b, s=5, m=20, tol=1e-11, max_restarts=3, basis="newton")
    checked = [(it, est) for it, est in g.estimates if it in ref and it > 20]
    assert len(checked) >= 4
    for it, est in checked:
        assert abs(est - ref[it]) <= 1e-9 * ref[it]


def test_leja_order_properties():
    rng = np.random.default_rng(0)
    re = rng.standard_normal(6)
    cz = rng.standard_normal(3) + 1j * np.abs(rng.standard_normal(3))
    theta = np.concatenate([re, cz, cz.conj()])
    order = krylov.leja_order(theta)
    assert len(order) == len(theta)
    assert abs(order[0]) == max(abs(z) for z in theta)
    for i, z in enumerate(order):                     # conjugates follow at once
        if z.imag > 0:
            assert order[i + 1] == z.conjugate()
    # greedy criterion: each point (first of a pair) maximises the product of its
    # distances to the points before it among the points still available
    for i in range(1, len(order)):
        if order[i].imag < 0:
            continue
        chosen, rest = order[:i], [z for z in order[i:] if z.imag >= 0]
        prod = lambda z: np.prod([abs(z - w) for w in chosen])  # noqa: E731
        assert prod(order[i]) >= max(prod(z) for z in rest) * (1 - 1e-12)


def test_newton_shifts_special_cases():
    # real spectrum: alpha = the eigenvalues in Leja order, beta = 0
    H = np.diag([1.0, -3.0, 2.0, 0.5])
    a, bt = krylov.newton_shifts(H, 4)
    assert list(a) == [-3.0, 2.0, 0.5, 1.0] or list(a) == [-3.0, 2.0, 1.0, 0.5]
    assert not bt.any()
    # a rotation-like 2 x 2 block: eigenvalues 2 +- 3i -> (Re, Re) and (0, Im^2)
    H = np.array([[2.0, -3.0], [3.0, 2.0]])
    a, bt = krylov.newton_shifts(H, 2)
    assert np.allclose(a, [2.0, 2.0]) and np.allclose(bt, [0.0, 9.0])
    # the pair cut by the last position keeps only its real part
    a, bt = krylov.newton_shifts(H, 1)
    assert np.allclose(a, [2.0]) and not bt.any()
    # zero shifts are the monomial basis
    Ahat = synth.laplace2d_csr(8).to_scipy()
    u = np.random.default_rng(1).standard_normal(Ahat.shape[0])
    assert np.array_equal(krylov.mpk_newton(Ahat, u, np.zeros(4), np.zeros(4)), krylov.mpk(Ahat, u, 4))
    # the recurrence v_{i+1} = (Ahat - alpha_i) v_i + beta_i v_{i-1} with a complex pair
    # gives the real polynomial (Ahat - Re)^2 + Im^2 applied to u
    V = krylov.mpk_newton(Ahat, u, np.array([0.7, 0.7]), np.array([0.0, 4.0]))
    D = Ahat.toarray()
    P = (D - 0.7 * np.eye(D.shape[0])) @ (D - 0.7 * np.eye(D.shape[0])) + 4.0 * np.eye(D.shape[0])
    assert np.allclose(V[:, 1], P @ u, rtol=1e-12, atol=1e-10)


def test_newton_basis_is_better_conditioned():
    # the reason for the Newton basis: its panels are far better conditioned than the
    # monomial ones at the same s
    A = synth.poisson3d_csr(12)
    Ahat, _ = krylov.jacobi_scaled(A)
    u = np.random.default_rng(3).standard_normal(Ahat.shape[0])
    u /= np.linalg.norm(u)
    # Ritz values of a 40-step Arnoldi on Ahat
    Q = np.zeros((Ahat.shape[0], 41))
    Hh = np.zeros((41, 40))
    Q[:, 0] = u
    for j in range(40):
        w = Ahat @ Q[:, j]
        for i in range(j + 1):
            Hh[i, j] = Q[:, i] @ w
            w -= Hh[i, j] * Q[:, i]
        Hh[j + 1, j] = np.linalg.norm(w)
        Q[:, j + 1] = w / Hh[j + 1, j]
    a, bt = krylov.newton_shifts(Hh[:40, :40], 10)
    cond = lambda V: np.linalg.cond(V / np.linalg.norm(V, axis=0))  # noqa: E731
    assert cond(krylov.mpk_newton(Ahat, u, a, bt)) < 1e-3 * cond(krylov.mpk(Ahat, u, 10))


def test_chebyshev_recurrence_is_scaled_chebyshev_polynomials():
    # the recurrence p_1 = z - c, p_2 = (z - c) p_1 - e2/2, p_{k+1} = (z - c) p_k - e2/4 p_{k-1}
    # reproduces 2 (e/2)^k T_k((z - c)/e), evaluated here with numpy's Chebyshev series
    # (complex e when the foci lie on the imaginary line)
    from numpy.polynomial import chebyshev as C
    z = np.linspace(-1.5, 3.5, 11)
    for lam in ([0.2, 1.9, 0.7, 1.1], [-1.0, 3.0, 0.5]):
        a, bt = krylov.chebyshev_shifts(np.diag(lam), 6)
        c, e = 0.5 * (max(lam) + min(lam)), 0.5 * (max(lam) - min(lam))
        # real spectrum: the ellipse is the interval [min, max] itself
        assert np.allclose(a, c, rtol=0, atol=1e-15) and np.isclose(-bt[1] * 2, e * e)
        V = krylov.mpk_newton(np.diag(z), np.ones_like(z), a, bt)
        for k in range(1, 7):
            ref = 2 * (e / 2) ** k * C.chebval((z - c) / e, [0] * k + [1])
            assert np.allclose(V[:, k - 1], ref, rtol=1e-12, atol=1e-12)
    # a single conjugate pair 2 +- 3i: a segment on the line Re z = 2 whose foci are
    # the pair itself (e2 = -9)
    a, bt = krylov.chebyshev_shifts(np.array([[2.0, -3.0], [3.0, 2.0]]), 4)
    assert np.allclose(a, 2.0) and np.allclose(bt, [0.0, 4.5, 2.25, 2.25])
    # complex points z = x + iy act as the real 2 x 2 blocks [[x, -y], [y, x]]; a real
    # polynomial p maps the block's first unit vector to (Re p(z), Im p(z))
    e = 3j
    zc = np.array([2 + 3j, 2 - 3j, 2.5 + 1j, 0.3 - 0.2j])
    D = np.zeros((8, 8))
    for i, zz in enumerate(zc):
        D[2 * i:2 * i + 2, 2 * i:2 * i + 2] = [[zz.real, -zz.imag], [zz.imag, zz.real]]
    u = np.tile([1.0, 0.0], 4)
    V = krylov.mpk_newton(D, u, a, bt)
    for k in range(1, 5):
        ref = 2 * (e / 2) ** k * C.chebval((zc - 2.0) / e, [0] * k + [1])
        assert np.allclose(V[0::2, k - 1], ref.real, rtol=1e-12, atol=1e-12)
        assert np.allclose(V[1::2, k - 1], ref.imag, rtol=1e-12, atol=1e-12)


def test_chebyshev_ellipse_closed_forms():
    # four corners c +- d +- iy: minimising a + y / sqrt(1 - d^2/a^2) gives
    # a^2 = d^2 + (y d^2)^(2/3); the unit-square corners give the circle of radius sqrt 2
    c, a, b = krylov.chebyshev_ellipse(np.array([1 + 1j, 1 - 1j, -1 + 1j, -1 - 1j]))
    assert c == 0.0 and abs(a - np.sqrt(2)) < 1e-14 and abs(b - np.sqrt(2)) < 1e-14
    for d, y in [(1.0, 0.5), (2.0, 0.1), (0.3, 2.0)]:
        pts = np.array([0.7 + d + 1j * y, 0.7 + d - 1j * y, 0.7 - d + 1j * y, 0.7 - d - 1j * y])
        c, a, b = krylov.chebyshev_ellipse(pts)
        assert abs(c - 0.7) < 1e-15
        assert abs(a * a - (d * d + (y * d * d) ** (2.0 / 3.0))) < 1e-13 * a * a
        assert abs((d / a) ** 2 + (y / b) ** 2 - 1.0) < 1e-13     # corners on the ellipse
    # a real spectrum with a vanishing conjugate pair tends to the interval (continuity)
    for eps in (1e-3, 1e-6, 1e-9):
        c, a, b = krylov.chebyshev_ellipse(np.array([0.1, 1.9, 1.9 + 1j * eps, 1.9 - 1j * eps]))
        assert abs(a - 0.9) < 10 * eps ** (2 / 3) and b < 10 * eps ** (1 / 3)


def test_chebyshev_ellipse_is_smallest_enclosing():
    # brute force over the family (centre c, axis-aligned semi-axes on a grid): no
    # ellipse that contains every Ritz value has a smaller capacity (a + b)/2, and the
    # returned ellipse contains every value
    rng = np.random.default_rng(5)
    for trial in range(10):
        re = rng.standard_normal(4)
        cz = rng.standard_normal(3) + 1j * rng.uniform(0.1, 2.0, 3)
        theta = np.concatenate([re, cz, cz.conj()])
        c, a, b = krylov.chebyshev_ellipse(theta)
        assert np.isclose(c, 0.5 * (theta.real.max() + theta.real.min()))
        x, y = theta.real - c, theta.imag
        assert np.all((x / a) ** 2 + (y / b) ** 2 <= 1 + 1e-9)
        top = 3 * max(np.abs(x).max(), np.abs(y).max())
        ga, gb = np.meshgrid(np.linspace(1e-3, top, 700), np.linspace(1e-3, top, 700))
        inside = np.ones(ga.shape, dtype=bool)
        for xi, yi in zip(x, y):
            inside &= (xi / ga) ** 2 + (yi / gb) ** 2 <= 1
        best = (ga + gb)[inside].min()
        assert best >= (a + b) * (1 - 1e-9)
        assert best <= (a + b) + 3 * top / 700


@pytest.mark.parametrize("nonsym", [False, True])
def test_chebyshev_estimates_equal_householder_gmres(nonsym):
    # the Chebyshev basis spans the same Krylov space: estimates equal Householder GMRES
    A = synth.convdiff2d_csr(24, seed=1)[0] if nonsym else synth.laplace2d_csr(20)
    b = synth.ones_rhs(A)
    ref = dict(krylov.householder_gmres(A, b, m=20, tol=1e-11, max_restarts=3).estimates)
    g = krylov.sstep_gmres(A, b, s=5, m=20, tol=1e-11, max_restarts=3, basis="chebyshev")
    checked = [(it, est) for it, est in g.estimates if it in ref and it > 20]
    assert len(checked) >= 2
    for it, est in checked:
        assert abs(est - ref[it]) <= 1e-9 * ref[it]


def test_chebyshev_basis_is_better_conditioned():
    A = synth.poisson3d_csr(12)
    Ahat, _ = krylov.jacobi_scaled(A)
    u = np.random.default_rng(3).standard_normal(Ahat.shape[0])
    u /= np.linalg.norm(u)
    Q = np.zeros((Ahat.shape[0], 41))
    Hh = np.zeros((41, 40))
    Q[:, 0] = u
    for j in range(40):
        w = Ahat @ Q[:, j]
        for i in range(j + 1):
            Hh[i, j] = Q[:, i] @ w
            w -= Hh[i, j] * Q[:, i]
        Hh[j + 1, j] = np.linalg.norm(w)
        Q[:, j + 1] = w / Hh[j + 1, j]
    a, bt = krylov.chebyshev_shifts(Hh[:40, :40], 10)
    cond = lambda V: np.linalg.cond(V / np.linalg.norm(V, axis=0))  # noqa: E731
    assert cond(krylov.mpk_newton(Ahat, u, a, bt)) < 1e-3 * cond(krylov.mpk(Ahat, u, 10))

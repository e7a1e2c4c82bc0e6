"""Pins of the oracle's block orthogonalization schemes against what the paper fixes:
O(eps) orthogonality and backward error (equations (1)-(3)), uniqueness of the QR
factorisation with non-negative diagonal (Figure 1 caption), the CholQR2 breakdown
beyond kappa ~ eps^{-1/2} (Section 5.1, Figure 4 caption) and its absence in the
randomized schemes (Propositions 5.2, 7.2), and textbook special cases."""
import numpy as np
import pytest

import synth
from oracle import metrics, orth
from oracle.dense import householder_qr
from oracle.sketch import Sketch

N0 = 20000


@pytest.fixture(scope="module")
def sk0():
    return Sketch(N0, 244, 8, 42)


@pytest.fixture(scope="module")
def V_k1e10():
    return synth.glued_blocks(N0, 12, 5, 1e10, seed=0)


def test_one_stage_rand_config0(V_k1e10, sk0):
    r = orth.block_orth_one_stage(V_k1e10, 5, sk0)
    assert r.ok
    assert metrics.orth_error(r.Q) <= 1e-13
    assert metrics.backward_error(V_k1e10, r.Q, r.R) <= 1e-14
    assert np.allclose(np.tril(r.R, -1), 0) and (np.diag(r.R) > 0).all()
    # per-block condition number is carried by R's diagonal blocks
    for j in range(12):
        Rjj = r.R[5 * j:5 * j + 5, 5 * j:5 * j + 5]
        assert 1e9 < metrics.cond2(Rjj) < 1e11


def test_cholqr2_breaks_down_on_config0(V_k1e10):
    r = orth.block_orth_cholqr2(V_k1e10, 5)
    assert not r.ok
    assert r.breakdown_block == 0 and r.breakdown_where.startswith("cholqr2")


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_cholqr2_fine_below_threshold(kappa, sk0):
    V = synth.glued_blocks(N0, 6, 5, kappa, seed=3)
    r = orth.block_orth_cholqr2(V, 5)
    assert r.ok and metrics.orth_error(r.Q) <= 1e-13
    assert metrics.backward_error(V, r.Q, r.R) <= 1e-14


def test_kappa_threshold_separates_cholqr2_from_rand(sk0):
    # Figure 4: CholQR2 fails once kappa(V_j) >= 1e8; RandCholQR keeps O(eps)
    for kappa, seed in [(1e9, 5), (1e12, 6), (1e14, 7)]:
        V = synth.glued_blocks(N0, 4, 5, kappa, seed=seed)
        assert not orth.block_orth_cholqr2(V, 5).ok
        r = orth.block_orth_one_stage(V, 5, sk0)
        assert r.ok and metrics.orth_error(r.Q) <= 1e-13
        assert metrics.backward_error(V, r.Q, r.R) <= 1e-14


@pytest.mark.parametrize("scheme", ["one", "two", "cholqr2"])
def test_R_matches_householder_reference(scheme, sk0):
    V = synth.glued_blocks(N0, 12, 5, 1e4, seed=1, v0=True)
    if scheme == "one":
        r = orth.block_orth_one_stage(V, 5, sk0, v0=True)
    elif scheme == "two":
        r = orth.block_orth_two_stage(V, 5, 30, sk0, v0=True)
    else:
        r = orth.block_orth_cholqr2(V, 5, v0=True)
    Qh, Rh = householder_qr(V, want_q=True)
    assert r.ok
    assert metrics.rel_diff(r.R, Rh) <= 1e-12
    assert np.abs(r.Q - Qh).max() <= 1e-10


@pytest.mark.parametrize("kappa", [1e4, 1e8, 1e12, 1e14])
def test_two_stage_orthogonality(kappa, sk0):
    V = synth.glued_blocks(N0, 12, 5, kappa, seed=11, v0=True)
    r = orth.block_orth_two_stage(V, 5, 30, sk0, v0=True)
    assert r.ok
    assert metrics.orth_error(r.Q) <= 1e-13
    assert metrics.backward_error(V, r.Q, r.R) <= 1e-14


def test_two_stage_big_panel_kappa_1e15():
    # Section 8, Figures 7-8 setup (scaled down in n): (m, s_hat, s) = (180, 60, 5)
    n = 20000
    V = synth.glued_blocks(n, 36, 5, 1e15, seed=21)
    sk = Sketch(n, 4 * 61, 8, 42)
    r = orth.block_orth_two_stage(V, 5, 60, sk)
    assert r.ok
    assert metrics.orth_error(r.Q) <= 1e-13
    assert metrics.backward_error(V, r.Q, r.R) <= 1e-14


def test_two_stage_with_s_hat_equal_s_is_one_stage(sk0):
    V = synth.glued_blocks(N0, 6, 5, 1e8, seed=4, v0=True)
    a = orth.block_orth_one_stage(V, 5, sk0, v0=True)
    b = orth.block_orth_two_stage(V, 5, 5, sk0, v0=True)
    assert np.allclose(a.Q, b.Q, rtol=0, atol=1e-13)
    assert metrics.rel_diff(b.R, a.R) <= 1e-13


def test_single_column_is_normalisation(sk0):
    v = np.random.default_rng(0).standard_normal((N0, 1))
    q, r = orth.cholqr(v)
    assert abs(r[0, 0] - np.linalg.norm(v)) <= 1e-14 * np.linalg.norm(v)
    assert np.allclose(q, v / np.linalg.norm(v), atol=1e-16)


def test_orthonormal_input_gives_identity_R(sk0):
    U, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((N0, 20)))
    for r in (orth.block_orth_one_stage(U, 5, sk0), orth.block_orth_two_stage(U, 5, 10, sk0)):
        assert r.ok
        assert np.abs(r.R - np.eye(20)).max() <= 1e-14
        assert np.abs(r.Q - U).max() <= 1e-14


def test_rand_hh_gives_well_conditioned_qbar(sk0):
    # Section 5.2: Qbar = V R_hat^{-1} has kappa = O(1) for numerically full-rank V
    V = synth.glued_blocks(N0, 1, 5, 1e12, seed=8)
    Qbar, Rh = orth.rand_hh(V, sk0)
    assert metrics.cond2(Qbar) < 10.0
    assert metrics.cond2(V) > 1e11


def test_mpk_laplace_basis_cholqr2_vs_rand():
    # Section 8, Figure 9 setting: v_{j+1} = A v_j on the 128^2 2D Laplacian,
    # v_1 = b/||b||, b = A*1.  CholQR2 breaks down once the basis is too
    # ill-conditioned; RandCholQR stays at O(eps) while the basis is full rank.
    A = synth.laplace2d_csr(128).to_scipy()
    b = A @ np.ones(A.shape[0])
    V = np.zeros((A.shape[0], 19))
    V[:, 0] = b / np.linalg.norm(b)
    for j in range(1, 19):
        V[:, j] = A @ V[:, j - 1]
        V[:, j] /= np.linalg.norm(V[:, j])
    sk = Sketch(A.shape[0], 84, 8, 42)
    first_fail = None
    for j in range(1, 19):
        W = V[:, :j + 1]
        try:
            orth.cholqr2(W)
        except orth.Breakdown:
            if first_fail is None:
                first_fail = j
        Q, R = orth.rand_cholqr(W, sk)
        assert metrics.orth_error(Q) <= 1e-13
    assert first_fail is not None
    assert metrics.cond2(V[:, :first_fail + 1]) > 1e7


# --- BCGS-PIP preprocessing (Section 7.1) -------------------------------------------
def test_bcgs_pip_first_panel_is_cholqr():
    # the section's footnote: with no earlier panel BCGS-PIP is CholQR
    V = synth.glued_blocks(3000, 1, 5, 1e3, seed=5)
    Qp, P, T = orth.bcgs_pip(np.zeros((3000, 0)), V)
    Qc, Rc = orth.cholqr(V)
    assert P.shape == (0, 5)
    assert np.array_equal(T, Rc) and np.array_equal(Qp, Qc)


def test_bcgs_pip_pythagorean_gram():
    # with an orthonormal Qbar, G - P^T P is the Gram of the projected block, so
    # T_jj^T T_jj = (Vh - Qbar P)^T (Vh - Qbar P) and Qbar_j is orthonormal and
    # orthogonal to Qbar
    rng = np.random.default_rng(3)
    Qbar, _ = np.linalg.qr(rng.standard_normal((4000, 10)))
    Vh = rng.standard_normal((4000, 5))
    Qj, P, T = orth.bcgs_pip(Qbar, Vh)
    W = Vh - Qbar @ (Qbar.T @ Vh)
    assert np.allclose(T.T @ T, W.T @ W, rtol=1e-12, atol=1e-10)
    assert np.allclose(P, Qbar.T @ Vh, rtol=0, atol=1e-12)
    assert metrics.orth_error(np.hstack([Qbar, Qj])) <= 1e-13
    assert np.allclose(Qj @ T + Qbar @ P, Vh, atol=1e-12)


def test_two_stage_pip_matches_householder_reference(sk0):
    V = synth.glued_blocks(N0, 12, 5, 1e4, seed=1, v0=True)
    r = orth.block_orth_two_stage(V, 5, 30, None, v0=True, preproc="pip")
    Qh, Rh = householder_qr(V, want_q=True)
    assert r.ok
    assert metrics.rel_diff(r.R, Rh) <= 1e-12
    assert metrics.orth_error(r.Q) <= 1e-13
    assert metrics.backward_error(V, r.Q, r.R) <= 1e-14


def test_two_stage_pip_breaks_down_where_rand_does_not(sk0):
    # Section 7.1: BCGS-PIP needs kappa(big panel)^2 eps < 1/2; RandBCGS2 only
    # kappa eps < 1/2 (Proposition 7.2).  kappa = 1e10 big panels: PIP breaks down,
    # the randomized preprocessing does not
    V = synth.glued_blocks(N0, 12, 5, 1e10, seed=2)
    pip = orth.block_orth_two_stage(V, 5, 30, None, preproc="pip")
    rand = orth.block_orth_two_stage(V, 5, 30, sk0)
    assert not pip.ok and pip.breakdown_where == "bcgs-pip"
    assert rand.ok and metrics.orth_error(rand.Q) <= 1e-13
    # below the threshold (kappa = 1e5, kappa^2 eps ~ 1e-6) PIP is O(eps)
    V = synth.glued_blocks(N0, 12, 5, 1e5, seed=2)
    pip = orth.block_orth_two_stage(V, 5, 30, None, preproc="pip")
    assert pip.ok and metrics.orth_error(pip.Q) <= 1e-13


def test_two_stage_pip_with_s_hat_equal_s_is_bcgs_cholqr():
    # one panel per big panel: preprocessing is CholQR, then CholQR + BCGS + CholQR,
    # i.e. BCGS2 with CholQR2 as the first intra-block step (same arithmetic)
    V = synth.glued_blocks(N0, 6, 5, 1e3, seed=4)
    a = orth.block_orth_two_stage(V, 5, 5, None, preproc="pip")
    b = orth.block_orth_cholqr2(V, 5)
    assert a.ok and b.ok
    assert np.allclose(a.Q, b.Q, rtol=0, atol=1e-12)
    assert metrics.rel_diff(a.R, b.R) <= 1e-12


@pytest.mark.parametrize("kind", ["gauss", "count_gauss"])
def test_rand_schemes_with_gaussian_sketches(kind):
    # Proposition 5.2 holds for any subspace embedding: RandCholQR with a Gaussian
    # (d = 2s per block; 2 s_hat for the big panels) or Count-Gauss map keeps
    # O(eps) orthogonality at kappa = 1e10 where CholQR2 fails, and the R factor
    # is the unique one of the Householder reference
    from oracle.sketch import CountGaussSketch, GaussianSketch
    n = 20000
    V = synth.glued_blocks(n, 12, 5, 1e10, seed=0)
    mk = (lambda d: GaussianSketch(n, d, 42)) if kind == "gauss" else \
         (lambda d: CountGaussSketch(n, d, 4 * d * d // 10, 42))
    one = orth.block_orth_one_stage(V, 5, mk(10))
    two = orth.block_orth_two_stage(V, 5, 30, mk(60))
    for r in (one, two):
        assert r.ok
        assert metrics.orth_error(r.Q) <= 1e-13
        assert metrics.backward_error(V, r.Q, r.R) <= 1e-14
    W = synth.glued_blocks(n, 12, 5, 1e4, seed=1)
    r = orth.block_orth_one_stage(W, 5, mk(10))
    _, Rh = householder_qr(W, want_q=True)
    assert metrics.rel_diff(r.R, Rh) <= 1e-12

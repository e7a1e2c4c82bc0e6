"""Pins of the oracle's learned-SPAI network: finite-difference gradients, the
Jacobi special case, the Frobenius form of the loss, first-order optimality of
the classical SPAI (Grote-Huckle) minimiser, and bfloat16 rounding."""
import numpy as np
import pytest

import synth
from oracle import gnn


@pytest.fixture(scope="module")
def small():
    A, _ = synth.convdiff2d_csr(12, seed=5)
    return A, gnn.Graph(A)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -2.5, 1e-30, 3.1415926])
    got = gnn.to_bf16(x)
    assert got[0] == 1.0
    assert got[1] == 1.0                      # tie -> even
    assert got[2] == 1.0 + 2**-7              # above the tie -> up
    assert got[3] == -2.5
    assert abs(got[5] - 3.140625) == 0.0      # pi in bf16
    assert np.all(np.abs(gnn.to_bf16(x[np.abs(x) > 1e-20]) - x[np.abs(x) > 1e-20])
                  <= 2**-8 * np.abs(x[np.abs(x) > 1e-20]))


def test_zero_weights_give_jacobi(small):
    A, G = small
    Mv = gnn.forward(np.zeros(gnn.n_params()), G)
    expect = np.where(G.row == G.col, 1.0 / G.diag[G.row], 0.0)
    assert np.array_equal(Mv, expect)


def test_loss_on_identity_is_frobenius(small):
    A, G = small
    theta = gnn.init_params(1)
    theta[-97:] = np.random.default_rng(2).standard_normal(97) * 0.01
    Mv = gnn.forward(theta, G)
    L, _ = gnn.loss_and_dM(Mv, G, np.eye(G.n))
    assert abs(L - gnn.frobenius_loss(A, Mv)) <= 1e-12 * L


def test_gradient_matches_finite_differences(small):
    A, G = small
    rng = np.random.default_rng(3)
    theta = gnn.init_params(4)
    theta[-97:] = rng.standard_normal(97) * 0.05
    Rb = rng.standard_normal((G.n, 4))
    L, g = gnn.loss_and_grad(theta, G, Rb, bf16=False)
    for k in rng.choice(len(theta), 40, replace=False):
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (gnn.loss_and_grad(tp, G, Rb, bf16=False)[0] - gnn.loss_and_grad(tm, G, Rb, bf16=False)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (k, fd, g[k])


def test_spai_is_the_frobenius_minimiser(small):
    A, G = small
    Ms = gnn.spai(A)
    L, dM = gnn.loss_and_dM(Ms, G, np.eye(G.n))
    jac = np.where(G.row == G.col, 1.0 / G.diag[G.row], 0.0)
    _, dJ = gnn.loss_and_dM(jac, G, np.eye(G.n))
    assert np.abs(dM).max() <= 1e-8 * np.abs(dJ).max()         # first-order optimality
    assert L < gnn.frobenius_loss(A, jac)
    rng = np.random.default_rng(6)
    for _ in range(3):
        assert L <= gnn.frobenius_loss(A, Ms + 1e-3 * rng.standard_normal(Ms.shape) * np.abs(Ms))


def test_adam_matches_definition():
    th = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    t1, m, v = gnn.adam_step(th, g, np.zeros(2), np.zeros(2), 1, lr=0.1)
    # first step of Adam moves each weight by lr * sign(g) (bias-corrected m/sqrt(v) = g/|g|)
    assert np.allclose(t1, th - 0.1 * np.sign(g), atol=1e-7)

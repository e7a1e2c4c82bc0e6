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


def _hand_graph_params():
    """Weights of the hand-computed example below: a few channels of width 32 are
    used, every value is exact in bfloat16."""
    p = {name: np.zeros(shp) for name, shp in gnn.param_shapes()}
    W = gnn.WIDTH
    # encoders: h ch0 = relu(row sum), h ch1 = relu(2 col sum);
    #           e ch2 = relu(-2 Ahat_ij), e ch3 = relu([i == j])
    p["Wn"][0, 0] = 1.0
    p["Wn"][1, 1] = 2.0
    p["We"][2, 0] = -2.0
    p["We"][3, 2] = 1.0
    # layer 0: m ch4 = relu(e2 + h_j0), m ch5 = relu(h_j1 - 1)
    #          h ch6 += relu(agg4 - h_i0), h ch0 += relu(agg5)
    p["Wm0"][4, 2] = 1.0
    p["Wm0"][4, W + 0] = 1.0
    p["Wm0"][5, W + 1] = 1.0
    p["bm0"][5] = -1.0
    p["Wh0"][6, W + 4] = 1.0
    p["Wh0"][6, 0] = -1.0
    p["Wh0"][0, W + 5] = 1.0
    # layer 1: m ch8 = relu(e4 + h_j6 - 2); h ch9 += relu(agg8 - h_i1)
    p["Wm1"][8, 4] = 1.0
    p["Wm1"][8, W + 6] = 1.0
    p["bm1"][8] = -2.0
    p["Wh1"][9, W + 8] = 1.0
    p["Wh1"][9, 1] = -1.0
    # layer 2: m ch10 = relu(1/2) on every edge; h ch7 += relu(agg10)
    p["bm2"][10] = 0.5
    p["Wh2"][7, W + 10] = 1.0
    # output: e8 + 2 e10 + h_i9 + h_i0 / 2 - h_j7 + 1/4 (+ [i == j])
    p["wo"][8] = 1.0
    p["wo"][10] = 2.0
    p["wo"][W + 9] = 1.0
    p["wo"][W + 0] = 0.5
    p["wo"][2 * W + 7] = -1.0
    p["bo"][0] = 0.25
    return gnn.flatten(p)


def test_forward_on_hand_computed_graph():
    """3 nodes, 7 stored entries (edges j -> i), every activation written out.

    A = [[2, -1, 0], [-2, 4, -1], [0, -1, 2]],  Ahat = D^-1 A:
      Ahat_01 = -1/2, Ahat_10 = -1/2, Ahat_12 = -1/4, Ahat_21 = -1/2.
    node features [sum_j |Ahat_ij|, sum_j |Ahat_ji|] (j != i):
      f0 = [1/2, 1/2], f1 = [3/4, 1], f2 = [1/2, 1/4]
    h0 (ch0, ch1): node0 (1/2, 1), node1 (3/4, 2), node2 (1/2, 1/2)
    e0 ch2 = relu(-2 Ahat_ij): e00 0, e01 1, e10 1, e11 0, e12 1/2, e21 1, e22 0;
    e0 ch3 = [i == j].
    layer 0, messages from h_j:  m ch4 = relu(e2 + h_j0), m ch5 = relu(h_j1 - 1)
      e00 (1/2, 0)  e01 (7/4, 1)  e10 (3/2, 0)  e11 (3/4, 1)  e12 (1, 0)
      e21 (7/4, 1)  e22 (1/2, 0)
      agg4: node0 9/4, node1 13/4, node2 9/4;  agg5: 1, 1, 1
      h ch6 = relu(agg4 - h0): 7/4, 5/2, 7/4;  h ch0 += 1: 3/2, 7/4, 3/2
    layer 1: m ch8 = relu(e4 + h_j6 - 2):
      e00 1/4, e01 9/4, e10 5/4, e11 5/4, e12 3/4, e21 9/4, e22 1/4
      agg8: node0 5/2, node1 13/4, node2 5/2
      h ch9 = relu(agg8 - h1): 3/2, 5/4, 2
    layer 2: m ch10 = 1/2 on every edge; agg10 = deg/2: 1, 3/2, 1; h ch7 = 1, 3/2, 1
    out_ij = e8 + 2 e10 + h_i9 + h_i0/2 - h_j7 + 1/4 + [i == j];  M_ij = out_ij / A_ii:
      e00 15/4 -> 15/8    e01 17/4 -> 17/8    e10 29/8 -> 29/32   e11 33/8 -> 33/32
      e12 25/8 -> 25/32   e21 19/4 -> 19/8    e22 17/4 -> 17/8
    """
    A = np.array([[2.0, -1.0, 0.0], [-2.0, 4.0, -1.0], [0.0, -1.0, 2.0]])
    G = gnn.Graph(A)
    assert list(zip(G.row.tolist(), G.col.tolist())) == [(0, 0), (0, 1), (1, 0), (1, 1), (1, 2),
                                                         (2, 1), (2, 2)]
    assert np.array_equal(G.f, [[0.5, 0.5], [0.75, 1.0], [0.5, 0.25]])
    assert np.array_equal(G.x, [[1, 1, 1], [-0.5, -0.5, 0], [-0.5, -0.5, 0], [1, 1, 1],
                                [-0.25, -0.5, 0], [-0.5, -0.25, 0], [1, 1, 1]])
    theta = _hand_graph_params()
    Mv, (_, cache) = gnn.forward(theta, G, keep=True)
    assert np.array_equal(Mv, [15 / 8, 17 / 8, 29 / 32, 33 / 32, 25 / 32, 19 / 8, 17 / 8])
    # intermediate activations of layer 0 (messages, aggregation input)
    zm0 = np.maximum(cache["zm0"], 0.0)
    assert np.array_equal(zm0[:, 4], [0.5, 1.75, 1.5, 0.75, 1.0, 1.75, 0.5])
    assert np.array_equal(zm0[:, 5], [0, 1, 0, 1, 0, 1, 0])
    assert np.array_equal(cache["v0"][:, gnn.WIDTH + 4], [2.25, 3.25, 2.25])
    assert np.array_equal(np.maximum(cache["zm1"], 0.0)[:, 8], [0.25, 2.25, 1.25, 1.25, 0.75, 2.25, 0.25])
    # final edge and node states entering the output layer
    q = cache["q"]
    W = gnn.WIDTH
    assert np.array_equal(q[:, 10], [0.5] * 7)
    assert np.array_equal(q[[0, 2, 5], W + 9], [1.5, 1.25, 2.0])          # h_i ch9
    assert np.array_equal(q[[0, 1, 4], 2 * W + 7], [1.0, 1.5, 1.0])       # h_j ch7

"""Pins of the oracle MLP of the learned screen (no GPU): the backpropagated
gradient equals central finite differences of the loss, and the loss equals
its definition evaluated from the forward pass."""
import numpy as np

import oracle


def _problem(seed, n=7):
    rng = np.random.default_rng(seed)
    w = rng.normal(size=oracle.MLP_WEIGHTS) * 0.3
    X = rng.normal(size=(n, 16))
    Y = rng.normal(size=n)
    return w, X, Y


def test_loss_is_its_definition():
    w, X, Y = _problem(1)
    y = oracle.mlp_forward(w, X)
    r = y - Y
    ref = np.mean(np.where(r < 0, 4.0, 1.0) * r * r)
    loss, _ = oracle.mlp_loss_grad(w, X, Y, 4.0)
    assert abs(loss - ref) <= 1e-14 * max(ref, 1.0)


def test_gradient_matches_central_differences():
    w, X, Y = _problem(2)
    loss, g = oracle.mlp_loss_grad(w, X, Y, 4.0)
    rng = np.random.default_rng(3)
    # every bias and a sample of weights of every layer, the output layer whole
    idx = np.unique(np.concatenate([rng.choice(oracle.MLP_WEIGHTS, 300, replace=False),
                                    np.arange(oracle.MLP_WEIGHTS - 65, oracle.MLP_WEIGHTS)]))
    h = 1e-6
    for e in idx:
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd = (oracle.mlp_loss_grad(wp, X, Y, 4.0)[0] - oracle.mlp_loss_grad(wm, X, Y, 4.0)[0]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * (1.0 + abs(g[e])), (e, fd, g[e])


def test_forward_of_a_hand_built_network():
    """A network built by hand in the documented weight layout (W1[16][64],
    b1, W2[64][64], b2, W3[64][64], b3, W4[64], b4; W[i][j] maps input i to
    unit j) whose output is known in closed form: two ReLU paths through
    off-diagonal weights, so a transposed or shifted layer changes the result."""
    w = np.zeros(oracle.MLP_WEIGHTS)
    o_b1 = 16 * 64
    o_W2 = o_b1 + 64
    o_b2 = o_W2 + 64 * 64
    o_W3 = o_b2 + 64
    o_b3 = o_W3 + 64 * 64
    o_W4 = o_b3 + 64
    o_b4 = o_W4 + 64
    assert o_b4 == oracle.MLP_WEIGHTS - 1
    # path A: x3 -> unit 5 -> unit 7 -> unit 9 = relu(4 - relu(x3)) -> 0.5 y
    w[3 * 64 + 5] = 1.0
    w[o_W2 + 5 * 64 + 7] = 1.0
    w[o_W3 + 7 * 64 + 9] = -1.0
    w[o_b3 + 9] = 4.0
    w[o_W4 + 9] = 0.5
    # path B: x0 - x1 + 0.5 -> unit 0 -> 2 * unit 63 -> unit 1 -> -1 y
    w[0 * 64 + 0] = 1.0
    w[1 * 64 + 0] = -1.0
    w[o_b1 + 0] = 0.5
    w[o_W2 + 0 * 64 + 63] = 2.0
    w[o_W3 + 63 * 64 + 1] = 1.0
    w[o_W4 + 1] = -1.0
    w[o_b4] = 0.125
    rng = np.random.default_rng(5)
    X = rng.normal(size=(50, 16)) * 3.0
    relu = lambda v: np.maximum(v, 0.0)  # noqa: E731
    expect = 0.5 * relu(4.0 - relu(X[:, 3])) - 2.0 * relu(X[:, 0] - X[:, 1] + 0.5) + 0.125
    assert np.max(np.abs(oracle.mlp_forward(w, X) - expect)) <= 1e-14
    # all-zero weights: the output bias alone
    z = np.zeros(oracle.MLP_WEIGHTS)
    z[o_b4] = -0.75
    assert np.all(oracle.mlp_forward(z, X) == -0.75)

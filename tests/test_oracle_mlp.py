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

"""Pins of the FP64 cost-model MLP reference (oracle/mlp.py): central finite
differences of its loss, and a one-unit network with a closed-form gradient."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, hidden, n = 5, 7, 9
    size = sum(i * o + o for i, o in mlp.shapes(n_in, hidden))
    p = rng.normal(scale=0.5, size=size)
    x = rng.normal(size=(n, n_in))
    t = rng.normal(size=n)
    loss, g = mlp.loss_and_grad(p, x, t, hidden)
    h = 1e-6
    for k in rng.choice(size, 60, replace=False):
        e = np.zeros(size)
        e[k] = h
        fd = (mlp.loss_and_grad(p + e, x, t, hidden)[0] - mlp.loss_and_grad(p - e, x, t, hidden)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_one_unit_network_closed_form():
    # hidden = 1, all weights positive: y = w4 relu(w3 relu(w2 relu(x w1 + b1) + b2) + b3) + b4
    x = np.array([[2.0]])
    t = np.array([0.0])
    p = np.array([0.5, 0.1, 2.0, 0.0, 3.0, 0.0, 4.0, 0.0])   # w1 b1 w2 b2 w3 b3 w4 b4
    a1 = 0.5 * 2 + 0.1
    y = 4.0 * 3.0 * 2.0 * a1
    loss, g = mlp.loss_and_grad(p, x, t, 1)
    assert abs(loss - y * y) < 1e-12
    d = 2 * y
    assert abs(g[7] - d) < 1e-12                      # d/db4
    assert abs(g[6] - d * 3.0 * 2.0 * a1) < 1e-12     # d/dw4
    assert abs(g[0] - d * 4 * 3 * 2 * 2.0) < 1e-12   # d/dw1 = d * w4 w3 w2 x

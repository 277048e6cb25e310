"""Pin for the FP64 schedule-MLP reference: its backpropagated gradient
matches central finite differences of its loss."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = rng.normal(0.0, 0.4, mlp.NPARAM)
    X = rng.uniform(0.0, 1.0, (40, mlp.NIN))
    Y = rng.normal(2.0, 1.0, 40)
    g = mlp.grad(w, X, Y)
    idx = rng.choice(mlp.NPARAM, size=120, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss(wp, X, Y) - mlp.loss(wm, X, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_layout():
    """A one-hot weight pattern routes input k to the output as the layout says."""
    w = np.zeros(mlp.NPARAM)
    o_w1, o_b1 = 0, mlp.H * mlp.NIN
    o_w2 = o_b1 + mlp.H
    o_b2 = o_w2 + mlp.H * mlp.H
    o_w3 = o_b2 + mlp.H
    o_b3 = o_w3 + mlp.H
    w[o_w1 + 5 * mlp.NIN + 2] = 3.0   # h1[5] = 3 * x[2]
    w[o_w2 + 7 * mlp.H + 5] = 2.0     # h2[7] = 2 * h1[5]
    w[o_w3 + 7] = 0.5                 # y = 0.5 * h2[7] + b3
    w[o_b3] = 1.0
    X = np.zeros((1, mlp.NIN))
    X[0, 2] = 0.25
    assert abs(mlp.forward(w, X)[0] - (1.0 + 0.5 * 2.0 * 3.0 * 0.25)) < 1e-15

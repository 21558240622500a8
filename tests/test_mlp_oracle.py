"""Pins of the emulator oracle: tabulated normal-CDF values and finite differences."""

import numpy as np

from oracle import mlp as OM


def test_gelu_tabulated():
    # g(z) = z Phi(z); Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208
    assert OM.gelu(np.array([0.0]))[0] == 0.0
    assert abs(OM.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(OM.gelu(np.array([-1.0]))[0] - (-1.0 * (1 - 0.8413447460685429))) < 1e-15
    assert abs(OM.gelu(np.array([2.0]))[0] - 2 * 0.9772498680518208) < 1e-15
    # derivative against a central difference
    z = np.linspace(-3, 3, 13)
    h = 1e-6
    fd = (OM.gelu(z + h) - OM.gelu(z - h)) / (2 * h)
    assert np.abs(fd - OM.gelu_grad(z)).max() < 1e-8


def _net(seed, n_in=3, width=8, depth=2):
    g = np.random.default_rng(seed)
    sizes = [n_in] + [width] * depth + [1]
    return [(g.standard_normal((sizes[i + 1], sizes[i])) / np.sqrt(sizes[i]), 0.1 * g.standard_normal(sizes[i + 1]))
            for i in range(len(sizes) - 1)]


def test_one_hidden_unit_by_hand():
    params = [(np.array([[2.0, -1.0]]), np.array([0.5])), (np.array([[3.0]]), np.array([-1.0]))]
    x = np.array([[1.0, 0.5]])
    y, _ = OM.forward(params, x, np.zeros(2), np.ones(2))
    z = 2.0 * 1.0 - 1.0 * 0.5 + 0.5                     # 2.0
    assert abs(y[0] - (3.0 * 2.0 * 0.9772498680518208 - 1.0)) < 1e-14
    assert z == 2.0


def test_gradients_finite_difference():
    params = _net(1)
    g = np.random.default_rng(2)
    x = g.uniform(-2, 2, (7, 3))
    t = g.standard_normal(7) * 3 + 1
    xs, xc, ys, yc = np.array([0.1, -0.2, 0.0]), np.array([0.5, 0.5, 1.0]), 1.0, 3.0
    loss, grads = OM.loss_and_grads(params, x, t, xs, xc, ys, yc)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for idx in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp = [(p[0].copy(), p[1].copy()) for p in params]
            Wm = [(p[0].copy(), p[1].copy()) for p in params]
            Wp[l][0][idx] += h
            Wm[l][0][idx] -= h
            fd = (OM.loss_and_grads(Wp, x, t, xs, xc, ys, yc)[0] - OM.loss_and_grads(Wm, x, t, xs, xc, ys, yc)[0]) / (2 * h)
            assert abs(fd - grads[l][0][idx]) <= 1e-7 * max(1.0, abs(fd))
        bp = [(p[0].copy(), p[1].copy()) for p in params]
        bm = [(p[0].copy(), p[1].copy()) for p in params]
        bp[l][1][0] += h
        bm[l][1][0] -= h
        fd = (OM.loss_and_grads(bp, x, t, xs, xc, ys, yc)[0] - OM.loss_and_grads(bm, x, t, xs, xc, ys, yc)[0]) / (2 * h)
        assert abs(fd - grads[l][1][0]) <= 1e-7 * max(1.0, abs(fd))

"""Pins for the FP64 surrogate-network oracle: the backward pass equals central differences of the
loss, and the forward pass of a hand-built network equals its closed form."""
import numpy as np

from oracle import mlp


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    p = mlp.init(seed=1)
    x = rng.uniform(-1, 1, (7, 4))
    t = rng.standard_normal((7, 4))
    loss, g = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(mlp.NPARAM, 200, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        num = (mlp.loss_and_grad(p + e, x, t)[0] - mlp.loss_and_grad(p - e, x, t)[0]) / (2 * h)
        assert abs(num - g[i]) < 1e-7 * max(1.0, abs(num)), (i, num, g[i])


def test_forward_closed_form():
    # one active path: x0 -> unit 0 -> unit 0 -> unit 0 -> output 0 with weights 1, biases 0
    layers = [(np.zeros((o, i)), np.zeros(o)) for o, i in mlp.SIZES]
    for W, _ in layers:
        W[0, 0] = 1.0
    p = mlp.pack(layers)
    x = np.array([[0.7, 0.1, -0.2, 0.3], [-1.3, 0, 0, 0]])
    y = mlp.forward(p, x)
    s = mlp.silu
    np.testing.assert_allclose(y[:, 0], s(s(s(x[:, 0]))), rtol=1e-15)
    np.testing.assert_allclose(y[:, 1:], 0.0)


def test_silu_grad():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    np.testing.assert_allclose(mlp.silu_grad(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-9)


def test_features_range():
    f = mlp.features([[0.5, -1.0, 4.0], [0, 0, 0]], 1.0, 2.0, 0.5, 2.0)
    np.testing.assert_allclose(f, [[1, 1, 1, 1], [-1, -1, -1, 1]])

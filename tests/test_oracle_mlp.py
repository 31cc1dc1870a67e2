"""Pins of the FP64 reference MLP (oracle/mlp.py): analytic gradients equal
central finite differences; a zero network outputs its last bias; the first
Adam step moves every parameter by lr against the gradient's sign."""
import numpy as np

from oracle import mlp


def _net(dims, seed):
    g = np.random.default_rng(seed)
    return [(g.standard_normal((dims[l + 1], dims[l])) * 0.5, g.standard_normal(dims[l + 1]) * 0.1)
            for l in range(len(dims) - 1)]


def test_gradients_equal_finite_differences():
    for dims in ((3, 1), (4, 5, 1), (5, 4, 3, 1)):
        params = _net(dims, sum(dims))
        g = np.random.default_rng(1)
        X = g.standard_normal((7, dims[0]))
        t = g.standard_normal(7)
        ana = mlp.gradients(params, X, t)
        num = mlp.numeric_gradients(params, X, t)
        for (aW, ab), (nW, nb) in zip(ana, num):
            assert np.allclose(aW, nW, rtol=1e-6, atol=1e-8)
            assert np.allclose(ab, nb, rtol=1e-6, atol=1e-8)


def test_zero_network_outputs_bias():
    params = [(np.zeros((3, 4)), np.zeros(3)), (np.zeros((1, 3)), np.array([0.7]))]
    y, _ = mlp.forward(params, np.ones((5, 4)))
    assert np.all(y == 0.7)


def test_first_adam_step_is_signed_lr():
    params = _net((3, 2, 1), 4)
    g = np.random.default_rng(2)
    X, t = g.standard_normal((9, 3)), g.standard_normal(9)
    grads = mlp.gradients(params, X, t)
    new = mlp.adam_step(params, grads, mlp.adam_state(params), lr=0.01)
    for (W, b), (W2, b2), (gW, gb) in zip(params, new, grads):
        assert np.allclose(W2 - W, -0.01 * np.sign(gW), atol=1e-7)
        assert np.allclose(b2 - b, -0.01 * np.sign(gb), atol=1e-7)


def test_adam_reduces_loss():
    params = _net((2, 8, 1), 5)
    g = np.random.default_rng(3)
    X = g.uniform(-1, 1, (64, 2))
    t = np.sin(X[:, 0]) + X[:, 1] ** 2
    st = mlp.adam_state(params)
    l0 = mlp.loss(params, X, t)
    for _ in range(300):
        params = mlp.adam_step(params, mlp.gradients(params, X, t), st, lr=0.01)
    assert mlp.loss(params, X, t) < 0.2 * l0

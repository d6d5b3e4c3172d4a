"""Pins of the cost-model MLP oracle: its analytic gradient against central finite
differences (an independent computation), and its packing/shape invariants."""
import numpy as np

from oracle import costmodel


def _data(n=37, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (n, costmodel.IN))
    t = rng.normal(0, 1, n)
    return X, t


def test_parameter_count_matches_library_constant():
    assert costmodel.NPARAM == 5313


def test_gradient_matches_central_differences():
    X, t = _data()
    p = costmodel.init(5).astype(np.float64)
    p += np.random.default_rng(1).normal(0, 0.05, p.size)  # biases off zero
    _, g = costmodel.loss_grad(p, X, t)
    rng = np.random.default_rng(2)
    idx = rng.choice(p.size, 120, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (costmodel.loss(p + e, X, t) - costmodel.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_linear_regime_closed_form():
    # with all pre-activations positive the network is affine: W3.W2.W1 x + const
    p = costmodel.unpack(costmodel.init(7).astype(np.float64))
    p["W1"] = np.abs(p["W1"])
    p["W2"] = np.abs(p["W2"])
    p["b1"][:] = 1.0
    p["b2"][:] = 1.0
    X = np.abs(_data()[0])
    y, _ = costmodel.forward(costmodel.pack(p), X)
    A = p["W3"] @ p["W2"] @ p["W1"]
    c = p["W3"] @ (p["W2"] @ p["b1"] + p["b2"]) + p["b3"][0]
    np.testing.assert_allclose(y, X @ A + c, rtol=1e-12, atol=1e-12)


def test_zero_residual_zero_gradient():
    X, _ = _data()
    p = costmodel.init(9).astype(np.float64)
    y, _ = costmodel.forward(p, X)
    loss, g = costmodel.loss_grad(p, X, y)
    assert loss == 0.0 and np.all(g == 0.0)

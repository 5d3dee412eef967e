"""Pins of the FP64 network reference (oracle/mlp_oracle.py) that the GPU
network kernels are checked against: finite differences, the constant
predictor, and the reduction to logistic regression."""
import numpy as np

from oracle import mlp_oracle as M


def _data(n=40, seed=1):
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.0, (n, M.NI))
    y = (rng.random(n) < 0.4).astype(np.float64)
    mean = rng.normal(0.0, 0.2, M.NI)
    scale = rng.uniform(0.5, 2.0, M.NI)
    return x, y, mean, scale


def test_backprop_matches_central_differences():
    x, y, mean, scale = _data()
    p = M.init_params(3)
    p[M.NI * M.NH:M.NI * M.NH + M.NH] = 0.05   # b1 away from zero
    g = M.grad(p, x, y, mean, scale)
    # every parameter group: W1, b1, W2, b2, w3, b3
    sizes = [M.NI * M.NH, M.NH, M.NH * M.NH, M.NH, M.NH, 1]
    o = np.cumsum([0] + sizes)
    idx = sorted({int(o[k]) + j for k in range(6) for j in (0, 7, 33) if j < sizes[k]})
    num = M.numeric_grad(p, x, y, mean, scale, idx=idx)
    for i, v in num.items():
        assert abs(g[i] - v) <= 1e-7 + 1e-6 * abs(v), (i, g[i], v)


def test_constant_predictor():
    x, y, mean, scale = _data(n=17)
    p = np.zeros(M.NPARAM)
    prob, _ = M.forward(p, x, mean, scale)
    assert np.all(prob == 0.5)
    assert abs(M.loss(p, x, y, mean, scale) - np.log(2.0)) < 1e-15
    g = M.grad(p, x, y, mean, scale)
    assert abs(g[-1] - np.mean(0.5 - y)) < 1e-15
    assert np.all(g[:-1] == 0.0)


def test_reduces_to_logistic_regression():
    """Positive inputs through identity layers: z = v . x + c, so the loss
    and gradient are those of logistic regression, sum (p - y) x / n."""
    rng = np.random.default_rng(5)
    n = 25
    x = rng.uniform(0.1, 1.0, (n, M.NI))
    y = (rng.random(n) < 0.5).astype(np.float64)
    v = rng.normal(0.0, 0.5, M.NI)
    c = 0.3
    W1 = np.zeros((M.NI, M.NH)); W1[:, :M.NI] = np.eye(M.NI)
    W2 = np.eye(M.NH)
    w3 = np.zeros(M.NH); w3[:M.NI] = v
    p = M.pack(W1, np.zeros(M.NH), W2, np.zeros(M.NH), w3, c)
    z = x @ v + c
    prob = 1.0 / (1.0 + np.exp(-z))
    want_loss = -np.mean(y * np.log(prob) + (1 - y) * np.log(1 - prob))
    assert abs(M.loss(p, x, y) - want_loss) < 1e-12
    g = M.grad(p, x, y)
    _, _, _, _, gw3, gb3 = M.unpack(g)
    np.testing.assert_allclose(gw3[:M.NI], x.T @ (prob - y) / n, rtol=1e-12, atol=1e-15)
    assert abs(gb3 - np.mean(prob - y)) < 1e-14

"""TEST INFRASTRUCTURE ONLY: the FP64 reference of the activation proposer's
network (the library's lbm_mlp_* entry points).  Only tests/ and the
benchmark's CPU legs use this module; the library never does.

The network is not part of the paper; it follows the definition in
include/lbm.h: a multilayer perceptron 34 -> 64 -> 64 -> 1 with ReLU hidden
layers, a logistic output and the mean binary cross-entropy, inputs
standardised as x' = (x - mean) * scale, parameters packed as W1 [34][64],
b1 [64], W2 [64][64], b2 [64], w3 [64], b3.  Written from those definitions
with numpy in float64: a forward pass, the gradient by backpropagation, and
central finite differences to check that gradient.
"""
from __future__ import annotations

import numpy as np

NI, NH = 34, 64
NPARAM = NI * NH + NH + NH * NH + NH + NH + 1


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (NPARAM,)
    o = 0
    W1 = p[o:o + NI * NH].reshape(NI, NH); o += NI * NH
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    w3 = p[o:o + NH]; o += NH
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, [b3]]).astype(np.float64)


def forward(params, x, mean=None, scale=None):
    """Probabilities and the intermediate values (xn, a1, h1, a2, h2, z)."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    x = np.asarray(x, dtype=np.float64)
    mean = np.zeros(NI) if mean is None else np.asarray(mean, dtype=np.float64)
    scale = np.ones(NI) if scale is None else np.asarray(scale, dtype=np.float64)
    xn = (x - mean) * scale
    a1 = xn @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    p = 1.0 / (1.0 + np.exp(-z))
    return p, (xn, a1, h1, a2, h2, z)


def loss(params, x, y, mean=None, scale=None):
    """Mean binary cross-entropy, -[y log p + (1 - y) log(1 - p)], written
    in terms of the logit z so that it stays finite."""
    _, (_, _, _, _, _, z) = forward(params, x, mean, scale)
    y = np.asarray(y, dtype=np.float64)
    return float(np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))))


def grad(params, x, y, mean=None, scale=None):
    """Gradient of the mean loss by backpropagation (chain rule layer by
    layer; dL/dz = (p - y) / n for the logistic output)."""
    W1, b1, W2, b2, w3, b3 = unpack(params)
    p, (xn, a1, h1, a2, h2, z) = forward(params, x, mean, scale)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    dz = (p - y) / n
    dw3 = h2.T @ dz
    db3 = dz.sum()
    dh2 = np.outer(dz, w3) * (a2 > 0)
    dW2 = h1.T @ dh2
    db2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (a1 > 0)
    dW1 = xn.T @ dh1
    db1 = dh1.sum(axis=0)
    return pack(dW1, db1, dW2, db2, dw3, db3)


def numeric_grad(params, x, y, mean=None, scale=None, h=1e-6, idx=None):
    """Central differences of the loss for the parameters in idx (all by
    default)."""
    p = np.array(params, dtype=np.float64)
    idx = range(NPARAM) if idx is None else idx
    out = {}
    for i in idx:
        old = p[i]
        p[i] = old + h
        lp = loss(p, x, y, mean, scale)
        p[i] = old - h
        lm = loss(p, x, y, mean, scale)
        p[i] = old
        out[i] = (lp - lm) / (2 * h)
    return out


def init_params(seed=0):
    """He-style random initialisation (for tests and training starts)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, np.sqrt(2.0 / NI), (NI, NH))
    W2 = rng.normal(0.0, np.sqrt(2.0 / NH), (NH, NH))
    w3 = rng.normal(0.0, np.sqrt(1.0 / NH), NH)
    return pack(W1, np.zeros(NH), W2, np.zeros(NH), w3, 0.0)

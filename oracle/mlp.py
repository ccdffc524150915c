"""FP64 reference of the learned-correction network: a multilayer perceptron
432 -> 256 -> 256 -> 121 with GELU activations, its mean-squared-error loss, the
gradients by manual backpropagation and one Adam step.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``): the GPU library
never imports it.  It is pinned in ``tests/test_oracle_mlp.py`` against central
finite differences of the loss and against a closed-form Adam step.

Parameter layout (one flat vector, the order the GPU library uses):
  W1 [H1 x I], b1 [H1], W2 [H2 x H1], b2 [H2], W3 [OP x H2], b3 [OP]
with OP = 128 >= O = 121 output rows; rows O..OP-1 of W3 and b3 are padding
and carry no loss.  y = W x + b row by row (x a row vector of features).

GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2,  GELU'(z) = Phi(z) + z phi(z).
Loss = sum over rows and the O real outputs of (out - target)^2 / (rows * O).
"""
from __future__ import annotations

import math

import numpy as np

I, H1, H2, O, OP = 432, 256, 256, 121, 128
SHAPES = [("W1", (H1, I)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)), ("W3", (OP, H2)), ("b3", (OP,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)

_erf = np.vectorize(math.erf, otypes=[np.float64])


def unpack(theta: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(parts: dict) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_prime(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta: np.ndarray, X: np.ndarray):
    """X [rows x I] -> (out [rows x OP], cache)."""
    P = unpack(theta)
    Z1 = X @ P["W1"].T + P["b1"]
    Y1 = gelu(Z1)
    Z2 = Y1 @ P["W2"].T + P["b2"]
    Y2 = gelu(Z2)
    out = Y2 @ P["W3"].T + P["b3"]
    return out, (X, Z1, Y1, Z2, Y2)


def loss(theta: np.ndarray, X: np.ndarray, T: np.ndarray) -> float:
    out, _ = forward(theta, X)
    d = out[:, :O] - T[:, :O]
    return float((d * d).sum() / (X.shape[0] * O))


def gradients(theta: np.ndarray, X: np.ndarray, T: np.ndarray):
    """(loss, flat gradient) by backpropagation through the three layers."""
    P = unpack(theta)
    out, (X, Z1, Y1, Z2, Y2) = forward(theta, X)
    rows = X.shape[0]
    d = out - T
    d[:, O:] = 0.0
    L = float((d[:, :O] ** 2).sum() / (rows * O))
    dO = 2.0 * d / (rows * O)
    g = {"W3": dO.T @ Y2, "b3": dO.sum(0)}
    dZ2 = (dO @ P["W3"]) * gelu_prime(Z2)
    g["W2"] = dZ2.T @ Y1
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ P["W2"]) * gelu_prime(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(0)
    return L, pack(g)


def adam_step(theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction at step t >= 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v

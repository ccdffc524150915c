"""Pins of the FP64 reference network (oracle/mlp.py), used to check the GPU
training kernels: backpropagated gradients against central finite differences
of the loss, GELU against its definition through the normal CDF, and one Adam
step against the update written out by hand for a scalar."""
import math

import numpy as np

import synth
from oracle import mlp


def _small_problem(seed):
    g = synth.rng(seed)
    theta = g.standard_normal(mlp.NPARAM) * 0.05
    X = g.standard_normal((6, mlp.I))
    T = g.standard_normal((6, mlp.OP))
    return theta, X, T


def test_gelu_against_normal_cdf():
    z = np.linspace(-6, 6, 101)
    phi_cdf = np.array([0.5 * math.erfc(-x / math.sqrt(2.0)) for x in z])
    assert np.allclose(mlp.gelu(z), z * phi_cdf, rtol=0, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_prime(z), fd, atol=1e-8)
    # limits: GELU(z) -> z for large z, -> 0 for very negative z
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12 and abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12


def test_backprop_against_finite_differences():
    theta, X, T = _small_problem(401)
    L, g = mlp.gradients(theta, X, T)
    assert abs(L - mlp.loss(theta, X, T)) < 1e-14
    rng = synth.rng(402)
    # a sample of coordinates in every block, and the padding rows of W3 / b3 (zero gradient)
    offs, k = [], 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        offs.extend((k + rng.choice(n, size=6, replace=False)).tolist())
        k += n
    h = 1e-6
    for i in offs:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])
    P = mlp.unpack(g)
    assert np.all(P["W3"][mlp.O:] == 0) and np.all(P["b3"][mlp.O:] == 0)


def test_adam_step_scalar_by_hand():
    theta, m, v = np.array([1.0]), np.array([0.0]), np.array([0.0])
    g = np.array([0.5])
    th, m, v = mlp.adam_step(theta, m, v, g, 1, 1e-3)
    # first step: m_hat = g, v_hat = g^2 -> theta - lr * g / (|g| + eps)
    assert abs(th[0] - (1.0 - 1e-3 * 0.5 / (0.5 + 1e-8))) < 1e-15
    th2, m2, v2 = mlp.adam_step(th, m, v, np.array([-0.25]), 2, 1e-3)
    mh = (0.9 * 0.05 + 0.1 * -0.25) / (1 - 0.81)
    vh = (0.999 * 0.00025 + 0.001 * 0.0625) / (1 - 0.999 ** 2)
    assert abs(th2[0] - (th[0] - 1e-3 * mh / (math.sqrt(vh) + 1e-8))) < 1e-15

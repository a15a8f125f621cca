"""Pins of the FP64 surrogate-network reference (oracle/mlp.py), CPU only.

- gelu against textbook values of the normal CDF and its symmetry
  gelu(-x) = gelu(x) - x; gelu' against central differences;
- the loss gradient against central differences of the loss itself, for every
  weight and bias tensor of a small network (catches a transposed operand, a
  dropped term or a wrong activation derivative);
- a network whose hidden pre-activations are driven far positive reduces to an
  affine map (gelu(z) -> z), compared with the explicit matrix product.
"""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_forms():
    # Phi(1) and Phi(2) of the standard normal distribution
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu(np.array([2.0]))[0] - 2 * 0.9772498680518208) < 1e-15
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    x = np.linspace(-4, 4, 33)
    np.testing.assert_allclose(mlp.gelu(-x), mlp.gelu(x) - x, atol=1e-15)


def test_gelu_grad_central_differences():
    x = np.linspace(-5, 5, 41)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, atol=1e-9)


def small_net(rng, dims=(7, 6, 5, 4), k_in=8):
    W, b = [], []
    kin = k_in
    for n in dims[1:]:
        W.append(rng.normal(0, 1.0 / math.sqrt(kin), size=(n, kin)))
        b.append(rng.normal(0, 0.2, size=n))
        kin = n
    W[0][:, dims[0]:] = 0.0
    return {"W": W, "b": b, "in_shift": rng.normal(size=dims[0]), "in_scale": rng.uniform(0.5, 2, size=dims[0]),
            "out_shift": rng.normal(size=dims[-1]), "out_scale": rng.uniform(0.5, 2, size=dims[-1])}


def test_loss_gradient_central_differences():
    rng = np.random.default_rng(0)
    p = small_net(rng)
    x = rng.normal(size=(9, 7))
    y = rng.normal(size=(9, 4))
    q, n_out = y.shape
    _, gW, gb = mlp.loss_and_grad(p, x, y)
    h = 1e-6
    for l in range(len(p["W"])):
        for tensor, grad in ((p["W"][l], gW[l]), (p["b"][l], gb[l])):
            fd = np.zeros_like(tensor)
            for idx in np.ndindex(tensor.shape):
                old = tensor[idx]
                tensor[idx] = old + h
                lp = mlp.loss_and_grad(p, x, y)[0]
                tensor[idx] = old - h
                lm = mlp.loss_and_grad(p, x, y)[0]
                tensor[idx] = old
                fd[idx] = (lp - lm) / (2 * h) / (q * n_out)
            np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-9)


def test_affine_limit():
    rng = np.random.default_rng(1)
    p = small_net(rng)
    for l in range(len(p["W"]) - 1):
        p["b"][l] = p["b"][l] + 60.0          # gelu(z) = z to machine precision for z > 40
        if l > 0:
            p["W"][l] = np.abs(p["W"][l])     # positive inputs stay positive
    x = rng.normal(size=(5, 7))
    y, _ = mlp.forward(p, x)
    a = np.zeros((5, 8))
    a[:, :7] = (x - p["in_shift"]) * p["in_scale"]
    for l in range(len(p["W"])):
        a = a @ p["W"][l].T + p["b"][l]
    np.testing.assert_allclose(y, a * p["out_scale"] + p["out_shift"], rtol=1e-12, atol=1e-12)

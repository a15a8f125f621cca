"""FP64 reference of the harmonic-surrogate network (test infrastructure only).

The surrogate is a plain multilayer perceptron: for layers l = 0..4,
z_l = W_l x_l + b_l, x_{l+1} = gelu(z_l) for l < 4, and the output is
y = z_4 * out_scale + out_shift.  The input x_0 is the 7 instance features
(offset field [T] x3, easy-axis theta and phi [rad], ln K, ln d) normalised as
(x - in_shift) * in_scale and zero-padded to 64.  gelu is the exact form
x * Phi(x) with Phi the standard normal CDF.

The training loss is the sum of squared errors in normalised output units,
sum (z_4 - (y - out_shift) / out_scale)^2; the gradients are those of that sum
divided by (queries * outputs).  Forward and backward are written out layer by
layer with NumPy in float64, the backward by the chain rule:
  dL/dz_4 = 2 (z_4 - t) / (q * n_out)
  dL/dW_l = (dL/dz_l)^T x_l,   dL/db_l = sum over queries of dL/dz_l
  dL/dz_{l-1} = (dL/dz_l W_l) * gelu'(z_{l-1}),  gelu'(x) = Phi(x) + x phi(x).
It is pinned in the CPU tests by finite differences of its own loss, by the
closed forms of gelu, and by a network that reduces to an affine map.
"""
import math

import numpy as np

_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def normalised_input(x, in_shift, in_scale, k_in=64):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((x.shape[0], k_in))
    out[:, :x.shape[1]] = (x - in_shift) * in_scale
    return out


def forward(params, x):
    """params: dict with W (list of [N_l][K_l]), b (list of [N_l]), in_shift,
    in_scale, out_shift, out_scale.  Returns (y, cache)."""
    W, b = params["W"], params["b"]
    a = normalised_input(x, params["in_shift"], params["in_scale"], W[0].shape[1])
    xs, zs = [a], []
    for l in range(len(W)):
        z = xs[-1] @ W[l].T + b[l]
        zs.append(z)
        if l < len(W) - 1:
            xs.append(gelu(z))
    y = zs[-1] * params["out_scale"] + params["out_shift"]
    return y, (xs, zs)


def loss_and_grad(params, x, y):
    """Sum of squared normalised errors and the gradients of (that sum / (q * n_out))."""
    W = params["W"]
    _, (xs, zs) = forward(params, x)
    t = (np.asarray(y, dtype=np.float64) - params["out_shift"]) / params["out_scale"]
    d = zs[-1] - t
    loss = float(np.sum(d * d))
    q, n_out = d.shape
    g = 2.0 * d / (q * n_out)
    gW, gb = [None] * len(W), [None] * len(W)
    for l in range(len(W) - 1, -1, -1):
        gW[l] = g.T @ xs[l]
        gb[l] = g.sum(axis=0)
        if l > 0:
            g = (g @ W[l]) * gelu_grad(zs[l - 1])
    return loss, gW, gb

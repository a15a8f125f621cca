"""Equilibrium references used as pins.

Test infrastructure (see ``oracle/__init__``).

* ``langevin`` -- the Langevin function of Eq. Langevin (Sec. 2.2, model M0):
  L_beta(z) = coth(beta z) - 1/(beta z); the equilibrium mean moment of an
  isotropic ensemble (K = 0) in a static field is L(xi) H/|H| with
  xi = beta |H| = bT |B|.
* ``boltzmann_mean`` -- brute-force quadrature of the Boltzmann density
  f ∝ exp(bT B.m + sigma (n.m)^2) on a fine latitude-longitude grid
  (Gauss-Legendre x trapezoid; spectrally accurate for this smooth density).
  It is the stationary state of Eq. FP-general in a static field.

Parity status: pinned by definition (closed form; direct quadrature).
"""
import numpy as np


def langevin(xi):
    xi = np.asarray(xi, dtype=np.float64)
    small = np.abs(xi) < 1e-4
    safe = np.where(small, 1.0, xi)
    val = 1.0 / np.tanh(safe) - 1.0 / safe
    return np.where(small, xi / 3.0 - xi ** 3 / 45.0, val)


def boltzmann_mean(bT, B, sigma, n, n_theta=400, n_phi=800):
    """<m> and <m m^T> of f ∝ exp(bT B.m + sigma (n.m)^2)."""
    x, w = np.polynomial.legendre.leggauss(n_theta)
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    s = np.sqrt(1 - x * x)
    m = np.stack([np.outer(s, np.cos(ph)), np.outer(s, np.sin(ph)), np.outer(x, np.ones(n_phi))], axis=-1)
    U = bT * (m @ np.asarray(B, dtype=np.float64)) + sigma * (m @ np.asarray(n, dtype=np.float64)) ** 2
    f = np.exp(U - U.max()) * w[:, None]
    Z = f.sum()
    mean = np.einsum("ij,ijc->c", f, m) / Z
    second = np.einsum("ij,ijc,ijd->cd", f, m, m) / Z
    return mean, second

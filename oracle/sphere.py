"""Real spherical harmonics, tangential gradients and sphere quadrature.

Test infrastructure (see ``oracle/__init__``).  The unknown density f of the
Fokker-Planck equation (Section 2.1, Eq. FP-general) lives on the unit sphere;
the oracle expands it in real orthonormal spherical harmonics up to degree L
(the paper's finite-volume mesh is not specified; this reading is recorded in
the design notes).

Convention (no Condon-Shortley phase):
    Y_{l,0}  = Q_l^0(cos t)
    Y_{l,m}  = sqrt(2) Q_l^m(cos t) cos(m p)       m > 0
    Y_{l,-m} = sqrt(2) Q_l^m(cos t) sin(m p)       m > 0
with Q_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m and P_l^m >= 0 near the
north pole for x -> 1^-, so Y_{1,1} ~ x, Y_{1,-1} ~ y, Y_{1,0} ~ z.
Flat index i = l*l + l + m.

Pinned by: orthonormality under quadrature, agreement with
``scipy.special.sph_harm_y`` (a library routine, CS phase converted), and a
central finite-difference check of the tangential gradient.
"""
import numpy as np


def n_coeffs(L):
    return (L + 1) * (L + 1)


def idx(l, m):
    return l * l + l + m


def lm_of(i):
    l = int(np.floor(np.sqrt(i)))
    return l, i - l * l - l


def _normalised_legendre(L, x):
    """Q[l, m, :] = normalised associated Legendre functions, m >= 0.

    Standard three-term recurrences for fully normalised functions."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    Q = np.zeros((L + 1, L + 1) + x.shape)
    Q[0, 0] = np.sqrt(1.0 / (4.0 * np.pi))
    for m in range(1, L + 1):
        Q[m, m] = Q[m - 1, m - 1] * np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s
    for m in range(0, L):
        Q[m + 1, m] = np.sqrt(2.0 * m + 3.0) * x * Q[m, m]
    for m in range(0, L + 1):
        for l in range(m + 2, L + 1):
            a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            Q[l, m] = a * (x * Q[l - 1, m] - b * Q[l - 2, m])
    return Q


def real_sh(L, theta, phi):
    """Y[i, ...] for all i < (L+1)^2 at polar angle theta, azimuth phi."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    Q = _normalised_legendre(L, np.cos(theta))
    Y = np.zeros((n_coeffs(L),) + theta.shape)
    r2 = np.sqrt(2.0)
    for l in range(L + 1):
        Y[idx(l, 0)] = Q[l, 0]
        for m in range(1, l + 1):
            Y[idx(l, m)] = r2 * Q[l, m] * np.cos(m * phi)
            Y[idx(l, -m)] = r2 * Q[l, m] * np.sin(m * phi)
    return Y


def real_sh_with_grad(L, theta, phi):
    """(Y, G) with G[i, ..., 3] the tangential gradient of Y_i in Cartesian
    components.  grad_S Y = e_t dY/dt + e_p (1/sin t) dY/dp; the theta
    derivative of Q_l^m uses (1-x^2) dP_l^m/dx = -l x P_l^m + (l+m) P_{l-1}^m.
    The points must avoid the poles (Gauss-Legendre nodes do)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    x = np.cos(theta)
    s = np.sin(theta)
    Q = _normalised_legendre(L, x)
    dQ = np.zeros_like(Q)                  # d/dtheta of Q_l^m
    for l in range(1, L + 1):
        for m in range(0, l + 1):
            prev = Q[l - 1, m] if m <= l - 1 else 0.0
            c = np.sqrt((2.0 * l + 1.0) / (2.0 * l - 1.0) * (l * l - m * m))
            dQ[l, m] = (l * x * Q[l, m] - c * prev) / s
    e_t = np.stack([x * np.cos(phi), x * np.sin(phi), -s], axis=-1)
    e_p = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=-1)
    N = n_coeffs(L)
    Y = np.zeros((N,) + theta.shape)
    G = np.zeros((N,) + theta.shape + (3,))
    r2 = np.sqrt(2.0)
    for l in range(L + 1):
        Y[idx(l, 0)] = Q[l, 0]
        G[idx(l, 0)] = dQ[l, 0][..., None] * e_t
        for m in range(1, l + 1):
            cm, sm = np.cos(m * phi), np.sin(m * phi)
            Y[idx(l, m)] = r2 * Q[l, m] * cm
            Y[idx(l, -m)] = r2 * Q[l, m] * sm
            G[idx(l, m)] = (r2 * dQ[l, m] * cm)[..., None] * e_t + \
                (r2 * Q[l, m] * (-m) * sm / s)[..., None] * e_p
            G[idx(l, -m)] = (r2 * dQ[l, m] * sm)[..., None] * e_t + \
                (r2 * Q[l, m] * m * cm / s)[..., None] * e_p
    return Y, G


def quadrature(n_theta, n_phi):
    """Tensor-product rule: Gauss-Legendre in cos(theta) x uniform (trapezoid)
    in phi.  Exact for every polynomial in (x, y, z) of degree
    <= min(2 n_theta - 1, n_phi - 1) restricted to the sphere.

    Returns theta, phi, weight (flattened) and the Cartesian points."""
    xg, wg = np.polynomial.legendre.leggauss(n_theta)
    ph = 2.0 * np.pi * np.arange(n_phi) / n_phi
    T, P = np.meshgrid(np.arccos(xg), ph, indexing="ij")
    W = np.outer(wg, np.full(n_phi, 2.0 * np.pi / n_phi))
    T, P, W = T.ravel(), P.ravel(), W.ravel()
    pts = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], axis=-1)
    return T, P, W, pts

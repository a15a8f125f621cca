"""Axially symmetric special case of Eq. FP-general, solved in 1-D.

Test infrastructure (see ``oracle/__init__``).

When the density does not depend on the azimuth about an axis a (field along
a and K = 0, or H = 0 and n = a), the precession terms of Eq. convection drop
out and with x = a.m the equation reduces to (textbook Smoluchowski form on
[-1, 1])

    df/dt = D d/dx [ (1 - x^2) ( df/dx - f dU/dx ) ],
    U(x) = bT B x        (field along a, K = 0)
    U(x) = sigma x^2     (H = 0, n = a)

which is expanded here in normalised Legendre polynomials
p_l = sqrt((2l+1)/2) P_l with the Galerkin matrix
    G_kl = -D int (1 - x^2) p_k' (p_l' - U' p_l) dx
evaluated by Gauss-Legendre quadrature (exact for these polynomial integrands).
This shares no code with ``sphere``/``galerkin``; the mean moment along a is
<x> = int x f dx * 2 pi / (2 pi) with f normalised to int f dx = 1.

Parity status: pinned (classical results: free diffusion rate 2D, small-barrier
Neel slope, Langevin stationary state).
"""
import numpy as np


def _legendre_and_derivative(L, x):
    """Normalised p_l(x) and p_l'(x) for l = 0..L."""
    P = np.zeros((L + 1,) + np.shape(x))
    dP = np.zeros_like(P)
    P[0] = 1.0
    if L >= 1:
        P[1] = x
        dP[1] = 1.0
    for l in range(2, L + 1):
        P[l] = ((2 * l - 1) * x * P[l - 1] - (l - 1) * P[l - 2]) / l
        dP[l] = dP[l - 2] + (2 * l - 1) * P[l - 1]
    norm = np.sqrt((2 * np.arange(L + 1) + 1) / 2.0)
    return P * norm[:, None], dP * norm[:, None]


def galerkin_1d(L, D, dU):
    """G with dc/dt = G c for f = sum_l c_l p_l; dU(x) the potential slope."""
    x, w = np.polynomial.legendre.leggauss(L + 4)
    p, dp = _legendre_and_derivative(L, x)
    q = (1 - x * x) * w
    return -D * np.einsum("kq,lq,q->kl", dp, dp - p * dU(x)[None, :], q)


def mean_x(c):
    """<x> = int x f dx for f = sum c_l p_l: only l = 1 contributes,
    int x p_1 dx = sqrt(2/3)."""
    return np.sqrt(2.0 / 3.0) * np.asarray(c)[..., 1]


def equilibrium(L, U, n_quad=400):
    """Projection of f ∝ exp(U(x)) on p_l, normalised to unit mass."""
    x, w = np.polynomial.legendre.leggauss(n_quad)
    p, _ = _legendre_and_derivative(L, x)
    f = np.exp(U(x) - np.max(U(x)))
    f /= np.sum(w * f)
    return p @ (w * f)

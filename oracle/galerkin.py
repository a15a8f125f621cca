"""Galerkin matrices of the Fokker-Planck operator, by quadrature of the weak form.

Test infrastructure (see ``oracle/__init__``).

Eq. FP-general:  df/dt = div(D grad f) - div(b f),   D = 1/(2 tau).
With f = sum_j c_j Y_j and orthonormal real Y_i, testing with Y_i and
integrating by parts on the closed sphere gives dc/dt = A c with

    A_ij = integral[ -D grad Y_i . grad Y_j + (b . grad Y_i) Y_j ] dm.

b (Eq. convection) is affine in the field, so A(t) = A0 + sum_k B_k(t) A_k:
A0 holds the diffusion and the two anisotropy terms, A_k the precession and
damping parts for a unit field along axis k (tesla).  Every matrix is
evaluated with a product quadrature that integrates the (polynomial)
integrand exactly, degree <= 2L + 2.  No closed-form coupling coefficient is
used anywhere in the oracle.

Parity status: pinned (conservation row, Langevin, Boltzmann quadrature,
free diffusion, Larmor precession, Neel small-barrier slope, rotation
covariance, 1-D Legendre special case).
"""
import numpy as np

from . import sphere
from .physics import drift


def weak_form_matrices(L, P, n):
    """Return (A0, A1) with A1[k] the field matrix of axis k (k = x, y, z)."""
    nt, nph = L + 4, 2 * L + 6
    T, Ph, W, pts = sphere.quadrature(nt, nph)
    Y, G = sphere.real_sh_with_grad(L, T, Ph)          # (N, Q), (N, Q, 3)
    zero = np.zeros(3)
    b0 = drift(pts, zero, n, P)                        # anisotropy part
    A0 = -P.D * sum((G[:, :, c] * W) @ G[:, :, c].T for c in range(3))
    A0 += (np.einsum("qc,iqc->iq", b0, G) * W) @ Y.T
    A1 = np.empty((3,) + A0.shape)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        bk = drift(pts, e, n, P) - b0                  # coefficient of B_k
        A1[k] = (np.einsum("qc,iqc->iq", bk, G) * W) @ Y.T
    return A0, A1


def boltzmann_coeffs(L, P, n, B, n_theta=120, n_phi=240):
    """SH projection of the Boltzmann density f ∝ exp(bT B.m + sigma (n.m)^2),
    normalised to unit mass, on a fine product grid.  This is the initial
    state chosen where the paper is silent (equilibrium at the field of t=0)
    and the stationary state of Eq. FP-general in a static field."""
    T, Ph, W, pts = sphere.quadrature(n_theta, n_phi)
    expo = P.bT * (pts @ np.asarray(B, dtype=np.float64)) + P.sigma * (pts @ n) ** 2
    f = np.exp(expo - expo.max())
    f /= np.sum(W * f)
    Y = sphere.real_sh(L, T, Ph)
    return Y @ (W * f)


def mean_moment(c):
    """<m> = integral m f dm (Eq. mean_magmom_FP divided by m0): only the
    l = 1 coefficients contribute; x, y, z = Y_{1,1}, Y_{1,-1}, Y_{1,0}
    times sqrt(4 pi / 3)."""
    s = np.sqrt(4.0 * np.pi / 3.0)
    c = np.asarray(c)
    return s * np.stack([c[..., 3], c[..., 1], c[..., 2]], axis=-1)

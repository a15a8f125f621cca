"""Physical constants, the drift field and the applied field.

Test infrastructure (see ``oracle/__init__``).

Units: every magnetic field is given as B = mu0*H in tesla (the paper writes
fields in T/mu0, Section 2 and Section 2.4).  With that choice mu0 cancels
from p1*H, p2*H and beta*H, so it never appears below.

Pinned by: free rotational diffusion (tau), the Langevin function and
Boltzmann quadrature (ratio of damping to diffusion, 2 sigma p1 = beta p3),
the Larmor precession of the mean moment (value and sense of p1), and the
small-barrier Neel relaxation slope (p4 against the diffusion).
"""
from dataclasses import dataclass
import numpy as np

K_BOLTZMANN = 1.380649e-23          # J/K, exact SI value


@dataclass(frozen=True)
class Material:
    """Section 2.4.1 / spec material: saturation magnetisation Ms [A/m],
    Gilbert damping alpha, gyromagnetic ratio gamma [rad/(s T)], temperature
    T_B [K]."""
    Ms: float = 474e3
    alpha: float = 0.1
    gamma: float = 1.76e11
    T_B: float = 293.0


@dataclass(frozen=True)
class Derived:
    V: float        # core volume V_C = pi d^3 / 6                      (Sec. 2.2, M0)
    m0: float       # V_C Ms                                            (Sec. 2.2, M0)
    gt: float       # gamma~ = gamma / (1 + alpha^2)                    (Sec. 2.1)
    tau: float      # V_C Ms / (2 kB T_B gamma~ alpha)                  (Sec. 2.1)
    D: float        # 1 / (2 tau), diffusion coefficient of Eq. FP-general
    p1: float       # gamma~ mu0      -> gamma~      for B in tesla     (Sec. 2.1)
    p2: float       # gamma~ alpha mu0 -> gamma~ alpha                  (Sec. 2.1)
    p3: float       # 2 gamma~ K / Ms                                   (Sec. 2.1)
    p4: float       # alpha p3                                          (Sec. 2.1)
    sigma: float    # K V_C / (kB T_B), anisotropy barrier
    bT: float       # beta / mu0 = m0 / (kB T_B), multiplies B in tesla  (Sec. 2.2, Eq. Langevin)


def derive(mat: Material, K: float, d: float) -> Derived:
    """Neel constants of Section 2.1 (paragraph after Eq. convection) and
    m0, beta, V_C of Section 2.2 (model M0)."""
    V = np.pi * d ** 3 / 6.0
    m0 = V * mat.Ms
    gt = mat.gamma / (1.0 + mat.alpha ** 2)
    kT = K_BOLTZMANN * mat.T_B
    tau = V * mat.Ms / (2.0 * kT * gt * mat.alpha)
    p3 = 2.0 * gt * K / mat.Ms
    return Derived(V=V, m0=m0, gt=gt, tau=tau, D=1.0 / (2.0 * tau),
                   p1=gt, p2=gt * mat.alpha, p3=p3, p4=mat.alpha * p3,
                   sigma=K * V / kT, bT=m0 / kT)


def drift(m, B, n, P: Derived):
    """Drift field b(m, H, n) of Eq. convection, for points m (..., 3) on the
    sphere, field B (3,) in tesla and easy axis n (3,):
        p1 H x m + p2 (m x H) x m + p3 (n.m) n x m + p4 (n.m) (m x n) x m."""
    m = np.asarray(m, dtype=np.float64)
    B = np.broadcast_to(np.asarray(B, dtype=np.float64), m.shape)
    n = np.broadcast_to(np.asarray(n, dtype=np.float64), m.shape)
    nm = np.sum(n * m, axis=-1, keepdims=True)
    return (P.p1 * np.cross(B, m)
            + P.p2 * np.cross(np.cross(m, B), m)
            + P.p3 * nm * np.cross(n, m)
            + P.p4 * nm * np.cross(np.cross(m, n), m))


def easy_axis(theta, phi):
    """n = (sin t cos p, sin t sin p, cos t).  The paper's in-plane angle
    vartheta of Section 2.2 (iii), n = (cos v, sin v, 0), is theta = pi/2,
    phi = vartheta."""
    return np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])


@dataclass(frozen=True)
class Drive:
    """Applied field H = H_SF + H_DF of Section 2 (selection field evaluated
    at a voxel = constant offset, Section 2.1 last paragraph).  Per axis k:
        B_k(t) = off_k + amp_k sin(2 pi freq_k t + phase_k)   [T]
    A cosine Lissajous drive (Section 1.1, Section 2.4) has phase pi/2."""
    amp: tuple
    freq: tuple
    phase: tuple
    period: float

    def field(self, t, off):
        t = np.asarray(t, dtype=np.float64)
        out = np.empty(t.shape + (3,))
        for k in range(3):
            out[..., k] = off[k] + self.amp[k] * np.sin(2.0 * np.pi * self.freq[k] * t + self.phase[k])
        return out

"""One Fokker-Planck instance -> mean-moment trace, its derivative and phi_hat.

Test infrastructure (see ``oracle/__init__``).

An instance is one (offset field at a voxel, easy axis n, anisotropy K, core
diameter d) tuple; the PDE has no spatial derivative (Section 2.1, last
paragraph), so each voxel offset is an independent solve.

Readings where the paper is silent (listed in the design notes):
* initial state = Boltzmann equilibrium at B(0) including the anisotropy;
* output samples t_j = (W + j / S) T, j = 0 .. P S - 1, for W warm-up periods,
  P output periods and S samples per period;
* d<m>/dt is exact: sqrt(4 pi/3) times the l = 1 rows of A(t_j) c(t_j);
* phi_hat_{p,k} = (1/S) sum_j (p . d<m>/dt)(t_j) exp(-2 pi i j k / S) over the
  last output period: the rectangle rule for the normalised signal of model
  M1 (Section 2.2), per unit m0, without the filter a_hat and the -mu0 c
  factors of Eq. MPI_model_fourier (those are fitted later by M1/M2).

Parity status: pinned through its parts (galerkin, radau) plus the drive
half-wave symmetry and the axially symmetric 1-D special case.
"""
from dataclasses import dataclass
import numpy as np

from . import galerkin
from .physics import Material, derive, easy_axis
from .radau import RadauIIA


@dataclass(frozen=True)
class Schedule:
    samples_per_period: int
    warmup_periods: int
    output_periods: int


@dataclass(frozen=True)
class Instance:
    h_off: tuple          # offset field B = mu0 H_SF(r) at the voxel [T]
    theta: float          # easy-axis polar angle
    phi: float            # easy-axis azimuth
    K: float              # anisotropy constant [J/m^3]
    d: float              # core diameter [m]
    L: int                # spherical-harmonic truncation degree


def sample_times(drive, sched):
    S = sched.samples_per_period
    j = np.arange(sched.output_periods * S)
    return (sched.warmup_periods + j / S) * drive.period


def solve_instance(mat: Material, drive, inst: Instance, sched: Schedule,
                   rtol=1e-12, ic_field=None, return_state=False):
    """Integrate Eq. FP-general for one instance; returns a dict with
    t, m (T x 3), dmdt (T x 3), and the integrator's step counts."""
    P = derive(mat, inst.K, inst.d)
    n = easy_axis(inst.theta, inst.phi)
    A0, A1 = galerkin.weak_form_matrices(inst.L, P, n)
    off = np.asarray(inst.h_off, dtype=np.float64)

    def A_of_t(t):
        B = drive.field(t, off)
        return A0 + B[0] * A1[0] + B[1] * A1[1] + B[2] * A1[2]

    B0 = drive.field(0.0, off) if ic_field is None else np.asarray(ic_field)
    c0 = galerkin.boltzmann_coeffs(inst.L, P, n, B0)
    t = sample_times(drive, sched)
    h_max = drive.period / sched.samples_per_period
    integ = RadauIIA(A_of_t, rtol=rtol, h0=min(h_max, 0.01 * P.tau), h_max=h_max)
    C = integ.integrate(0.0, c0, t)
    m = galerkin.mean_moment(C)
    dC = np.stack([A_of_t(tj) @ cj for tj, cj in zip(t, C)])
    dmdt = galerkin.mean_moment(dC)
    out = dict(t=t, m=m, dmdt=dmdt, steps=integ.n_steps, rejected=integ.n_rejected)
    if return_state:
        out["c"] = C
    return out


def phi_hat(dmdt, channels, samples_per_period, k_max):
    """phi_hat[p, k] (complex) over the last full period of dmdt (T x 3) for
    receive directions channels (C x 3), k = 0..k_max."""
    S = samples_per_period
    u = np.asarray(dmdt)[-S:] @ np.asarray(channels, dtype=np.float64).T     # (S, C)
    j = np.arange(S)
    k = np.arange(k_max + 1)
    E = np.exp(-2j * np.pi * np.outer(k, j) / S)                             # (K, S)
    return (E @ u).T / S

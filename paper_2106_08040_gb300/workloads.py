"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

Only input generation lives here (voxel grids, drive settings, parameter
draws); none of the method's arithmetic.  The shapes follow the paper's
experimental setting (Sec. 2.4: Lissajous drive f_x = 2.5 MHz/102,
f_y = 2.5 MHz/96, 1632 samples per 652.8 us period at 2.5 MHz, selection
gradient (-1, -1, 2) T/mu0/m, 2D voxel grid of offsets; Sec. 2.4.1 parameter
grids) at the sizes of the benchmark workloads below.
"""
from dataclasses import dataclass

import numpy as np

INSTANCE_FIELDS = [("h_off", "<f8", (3,)), ("theta", "<f8"), ("phi", "<f8"), ("K", "<f8"),
                   ("d", "<f8"), ("L", "<i4"), ("flags", "<i4")]
INSTANCE_DTYPE = np.dtype(INSTANCE_FIELDS)

SEED = 20210615


@dataclass(frozen=True)
class DriveSpec:
    amp: tuple
    freq: tuple
    phase: tuple
    period: float
    samples_per_period: int
    warmup_periods: int
    output_periods: int


def drive_sin1d(f=25e3, amp=0.012, periods=4, samples=1000):
    """1-D sinusoidal drive along x (single-instance workload)."""
    return DriveSpec(amp=(amp, 0.0, 0.0), freq=(f, f, f), phase=(0.0, 0.0, 0.0), period=1.0 / f,
                     samples_per_period=samples, warmup_periods=0, output_periods=periods)


def drive_lissajous(amp=0.012, warmup=1, periods=1):
    """Cosine Lissajous drive of Sec. 2.4 (12 mT per axis here)."""
    fx, fy = 2.5e6 / 102.0, 2.5e6 / 96.0
    return DriveSpec(amp=(amp, amp, 0.0), freq=(fx, fy, 0.0), phase=(np.pi / 2, np.pi / 2, 0.0),
                     period=1632 / 2.5e6, samples_per_period=1632, warmup_periods=warmup,
                     output_periods=periods)


def make_instances(n):
    a = np.zeros(n, dtype=INSTANCE_DTYPE)
    return a


def voxel_offsets(nx, ny, fov=24e-3, gradient=(-1.0, -1.0, 2.0), z=0.0):
    """Offset fields B = G r [T] at the cell centres of an nx x ny grid on a
    fov x fov plane at height z; instance index = iy * nx + ix."""
    xs = -fov / 2 + (np.arange(nx) + 0.5) * fov / nx
    ys = -fov / 2 + (np.arange(ny) + 0.5) * fov / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")          # [iy, ix]
    off = np.stack([gradient[0] * X.ravel(), gradient[1] * Y.ravel(), np.full(X.size, gradient[2] * z)], axis=1)
    return off


def single_instance_workload():
    """1 instance: zero offset, easy axis at 45 deg in the x-y plane, K = 2e3 J/m^3,
    d = 20 nm, L = 10; 4 periods of a 25 kHz, 12 mT sinusoidal drive along x,
    1000 samples per period."""
    inst = make_instances(1)
    inst["theta"] = np.pi / 2
    inst["phi"] = np.pi / 4
    inst["K"] = 2e3
    inst["d"] = 20e-9
    inst["L"] = 10
    return drive_sin1d(), inst


def system_matrix_workload(nx=32, ny=32, L=16):
    """System-matrix batch: nx x ny voxels on 24 x 24 mm, gradient
    diag(-1, -1, 2) T/m, easy axis along x, K = 2e3 J/m^3, d = 20 nm; cosine
    Lissajous drive, 1 warm-up + 1 output period of 1632 samples."""
    inst = make_instances(nx * ny)
    inst["h_off"] = voxel_offsets(nx, ny)
    inst["theta"] = np.pi / 2
    inst["phi"] = 0.0
    inst["K"] = 2e3
    inst["d"] = 20e-9
    inst["L"] = L
    return drive_lissajous(), inst


def random_instances(n, L, seed=SEED, max_offset=0.012, K_range=(5e2, 1e4), d_median=20e-9, d_sigma=0.1):
    """Seeded random instances (offsets uniform in a cube, easy axes uniform on
    the sphere, K log-uniform, d log-normal)."""
    rng = np.random.default_rng(seed)
    inst = make_instances(n)
    inst["h_off"] = rng.uniform(-max_offset, max_offset, size=(n, 3))
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    inst["theta"] = np.arccos(np.clip(v[:, 2], -1, 1))
    inst["phi"] = np.arctan2(v[:, 1], v[:, 0])
    inst["K"] = np.exp(rng.uniform(np.log(K_range[0]), np.log(K_range[1]), size=n))
    inst["d"] = d_median * np.exp(d_sigma * rng.normal(size=n))
    inst["L"] = L
    return inst


def fibonacci_directions(n=16):
    """n easy-axis directions from the Fibonacci sphere: z_i = 1 - (2i + 1)/n,
    azimuth i * pi * (3 - sqrt(5)); returns (theta, phi) arrays."""
    i = np.arange(n)
    z = 1.0 - (2 * i + 1) / n
    theta = np.arccos(z)
    phi = np.mod(i * np.pi * (3.0 - np.sqrt(5.0)), 2 * np.pi)
    return theta, phi


def uneven_sweep_instances(n, L, seed=SEED, nxy=64, fov=24e-3, n_dir=16, K_range=(5e2, 1e4), d_median=20e-9,
                           d_sigma=0.1):
    """n random draws from the uneven-sweep distribution: a voxel of the nxy x nxy
    grid on the z = 0 plane (gradient diag(-1, -1, 2) T/m over fov), one of
    n_dir Fibonacci easy-axis directions, K log-uniform over K_range, d
    log-normal (median d_median, log-sd d_sigma); truncation degree L
    (scalar or array)."""
    rng = np.random.default_rng(seed)
    inst = make_instances(n)
    off = voxel_offsets(nxy, nxy, fov=fov)
    inst["h_off"] = off[rng.integers(0, nxy * nxy, size=n)]
    th, ph = fibonacci_directions(n_dir)
    k = rng.integers(0, n_dir, size=n)
    inst["theta"] = th[k]
    inst["phi"] = ph[k]
    inst["K"] = np.exp(rng.uniform(np.log(K_range[0]), np.log(K_range[1]), size=n))
    inst["d"] = d_median * np.exp(d_sigma * rng.normal(size=n))
    inst["L"] = L
    return inst


def high_degree_workload(L):
    """One instance resolved only at high truncation degree (barrier sigma ~ 11,
    d = 22 nm, K = 8e3 J/m^3, easy axis (1.1, 0.4) rad, offset (2, -3, 1) mT)
    under a 12 mT, 50 kHz drive along x, one period of 64 samples, degree L."""
    dspec = DriveSpec(amp=(0.012, 0.0, 0.0), freq=(50e3, 50e3, 50e3), phase=(0.0, 0.0, 0.0),
                      period=2e-5, samples_per_period=64, warmup_periods=0, output_periods=1)
    inst = make_instances(1)
    inst["h_off"] = [[0.002, -0.003, 0.001]]
    inst["theta"], inst["phi"] = 1.1, 0.4
    inst["K"], inst["d"] = 8e3, 22e-9
    inst["L"] = L
    return dspec, inst

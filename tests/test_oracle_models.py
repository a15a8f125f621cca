"""Pins of oracle/models.py (Section 2.2 models M0, M1, M2; Section 2.3
distance measures) against closed forms, library routines and brute force."""
import mpmath
import numpy as np
import pytest

from oracle import models, physics


def test_langevin_values_and_series_branch():
    """Eq. Langevin at high-precision reference values, on both sides of the
    series threshold, for real and complex arguments."""
    mpmath.mp.dps = 40
    for x in (1e-6, 5e-3, 0.0201, 0.3, 0.4999, 0.5001, 1.0, 7.5, 40.0):
        ref = float(mpmath.coth(x) - 1 / mpmath.mpf(x))
        assert abs(models.langevin_c(x) - ref) <= 2e-15 * abs(ref), x
    assert models._LSER[:4] == [1 / 3, -1 / 45, 2 / 945, -1 / 4725]
    z = 0.25 + 0.004j
    ref = complex(mpmath.coth(mpmath.mpc(z.real, z.imag)) - 1 / mpmath.mpc(z.real, z.imag))
    assert abs(models.langevin_c(z) - ref) <= 1e-15 * abs(ref)


def test_equilibrium_moment_limits():
    """|m| -> xi/3 for a weak field, 1 - 1/xi for a strong one; parallel to B."""
    P = physics.derive(physics.Material(), 0.0, 20e-9)
    B = np.array([1e-7, 2e-7, -1e-7])
    m = models.equilibrium_moment(P.bT, B)
    np.testing.assert_allclose(m, P.bT * B / 3.0, rtol=1e-9)
    B = np.array([0.0, 0.3, 0.4])                  # |B| = 0.5 T, xi ~ 245
    m = models.equilibrium_moment(P.bT, B)
    xi = P.bT * 0.5
    np.testing.assert_allclose(np.linalg.norm(m), 1.0 / np.tanh(xi) - 1.0 / xi, rtol=1e-14)
    np.testing.assert_allclose(np.cross(m, B), 0.0, atol=1e-14)


def test_equilibrium_derivative_matches_central_differences():
    """Complex-step d<m>/dt of model M0 against a 4th-order central difference
    of the trace itself, through a field zero crossing (voxel at the centre)."""
    drv = physics.Drive(amp=(0.012, 0.012, 0.0), freq=(2.5e6 / 102, 2.5e6 / 96, 0.0),
                        phase=(np.pi / 2, np.pi / 2, 0.0), period=1632 / 2.5e6)
    t = np.linspace(0.0, drv.period, 97)
    for off in ((0.0, 0.0, 0.0), (0.004, -0.002, 0.001)):
        m, dm = models.equilibrium_trace(physics.Material(), drv, 20e-9, off, t)
        h = 1e-3 * drv.period / 1632
        mm = [models.equilibrium_trace(physics.Material(), drv, 20e-9, off, t + s * h)[0] for s in (-2, -1, 1, 2)]
        fd = (mm[0] - 8 * mm[1] + 8 * mm[2] - mm[3]) / (12 * h)
        assert np.abs(fd - dm).max() <= 1e-6 * np.abs(dm).max()


def test_equilibrium_static_field_has_no_derivative():
    drv = physics.Drive(amp=(0.0, 0.0, 0.0), freq=(1e4, 1e4, 1e4), phase=(0.0, 0.0, 0.0), period=1e-4)
    m, dm = models.equilibrium_trace(physics.Material(), drv, 20e-9, (0.003, 0.0, 0.0), np.linspace(0, 1e-4, 9))
    assert np.abs(dm).max() == 0.0
    P = physics.derive(physics.Material(), 0.0, 20e-9)
    np.testing.assert_allclose(m[:, 0], models.langevin_c(P.bT * 0.003), rtol=1e-15)


def _rand_complex(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_m1_fit_is_the_least_squares_solution():
    """a_k against a library least-squares solve of min_a ||a Phi_k - S_k||_2
    per row; a planted filter is recovered with zero row error."""
    rng = np.random.default_rng(3)
    N, C, K = 37, 2, 11
    Phi = _rand_complex(rng, (N, C, K))
    S = _rand_complex(rng, (N, C, K))
    a, eps = models.m1_fit(Phi, S)
    for c in range(C):
        for k in range(K):
            sol = np.linalg.lstsq(Phi[:, c, k][:, None], S[:, c, k], rcond=None)[0][0]
            assert abs(sol - a[c, k]) <= 1e-13 * abs(sol)
            r = S[:, c, k] - sol * Phi[:, c, k]
            ref = np.sqrt(np.mean(np.abs(r) ** 2)) / np.abs(S[:, c, k]).max()
            assert abs(eps[c, k] - ref) <= 1e-13 * ref
    a_true = _rand_complex(rng, (C, K))
    a2, eps2 = models.m1_fit(Phi, a_true[None] * Phi)
    np.testing.assert_allclose(a2, a_true, rtol=1e-13)
    assert eps2.max() <= 1e-14


def test_eps_row_special_cases():
    """Eq. error1: zero model -> RMS / max of the row; constant rows -> |c - d| / |c|."""
    rng = np.random.default_rng(4)
    S = _rand_complex(rng, (50, 1, 3))
    e = models.eps_row(S, np.zeros_like(S))
    np.testing.assert_allclose(e, np.sqrt(np.mean(np.abs(S) ** 2, 0)) / np.abs(S).max(0), rtol=1e-15)
    c, d = 2.0 - 1.0j, 1.5 + 0.5j
    e = models.eps_row(np.full((9, 1, 1), c), np.full((9, 1, 1), d))
    assert abs(e[0, 0] - abs(c - d) / abs(c)) <= 1e-15


def test_mixing_orders_by_brute_force():
    """Eq. mix with N_dens = 16 (Section 2.4): the excitation frequencies are
    k(1,0) = 16 and k(0,1) = 17; every decomposition satisfies Eq. mix and no
    pair in a box of the same equation has a smaller |m_x| + |m_y|."""
    nd = 16
    assert models.mixing_order(16, nd) == (1, 0)
    assert models.mixing_order(17, nd) == (0, 1)
    assert models.mixing_order(0, nd) == (0, 0)
    for k in range(0, 817):
        mx, my = models.mixing_order(k, nd)
        assert mx * nd + my * (nd + 1) == k
        best = min(abs(a) + abs(b) for a in range(-60, 61) for b in range(-60, 61) if a * nd + b * (nd + 1) == k)
        assert abs(mx) + abs(my) == best


def test_freq_index_set_and_global_measure():
    ks = models.freq_index_set(3, 2, 16)
    assert 0 not in ks and 16 not in ks and 17 not in ks
    assert len(ks) == 4 * 3 - 3
    eps = np.full((2, 2, 100), 0.25)
    assert abs(models.eps_global(eps, ks) - 0.25) <= 1e-15
    eps[1, :, ks[0]] = 0.0
    ef = models.eps_freq(eps)
    assert abs(ef[ks[0]] - 0.25 / np.sqrt(2)) <= 1e-15


def _m2_dictionary(rng, A=3, J=6, N=40, C=2, K=12):
    Psi = [[_rand_complex(rng, (N, C, K)) for _ in range(J)] for _ in range(A)]
    return Psi


def test_m2_recovers_planted_weights():
    """An exact non-negative superposition of the dictionary is recovered
    with zero residual (full rank), and a TSVD fit at full rank equals it."""
    rng = np.random.default_rng(5)
    Psi = _m2_dictionary(rng)
    w_true = np.array([0.0, 1.5, 0.0, 0.25, 2.0, 0.0])
    S = [sum(w * p for w, p in zip(w_true, Pa)) for Pa in Psi]
    ks = np.arange(1, 12)
    w, res, sv, _ = models.m2_weights(Psi, S, ks)
    np.testing.assert_allclose(w, w_true, atol=1e-10)
    assert res <= 1e-10
    w6, res6, _, _ = models.m2_weights(Psi, S, ks, s_rank=6)
    np.testing.assert_allclose(w6, w_true, atol=1e-9)


def test_m2_solution_satisfies_the_kkt_conditions():
    """Noisy data: the NNLS weights satisfy the optimality conditions of the
    quadratic program min 1/2 w^T A w + f^T w, w >= 0 (A = Re M^H M,
    f = -Re M^H y): w >= 0, gradient >= 0, and w_j * gradient_j = 0."""
    rng = np.random.default_rng(6)
    Psi = _m2_dictionary(rng)
    S = [_rand_complex(rng, Psi[0][0].shape) for _ in Psi]
    ks = np.arange(12)
    w, res, sv, _ = models.m2_weights(Psi, S, ks)
    cols, ys = [], []
    for Pa, Sa in zip(Psi, S):
        sig = 1.0 / np.abs(Sa).max(0)
        ys.append((sig * Sa).reshape(-1))
        cols.append(np.stack([(sig * p).reshape(-1) for p in Pa], 1))
    M, y = np.concatenate(cols), np.concatenate(ys)
    M2, y2 = models.m2_matrix(Psi, S, ks)
    np.testing.assert_array_equal(M, M2)
    np.testing.assert_array_equal(y, y2)
    A = np.real(np.conj(M.T) @ M)
    f = -np.real(np.conj(M.T) @ y)
    g = A @ w + f
    scale = np.abs(A).max() * max(1.0, np.abs(w).max())
    assert (w >= 0).all()
    assert (g >= -1e-9 * scale).all()
    assert np.abs(w * g).max() <= 1e-9 * scale * max(1.0, np.abs(w).max())
    assert abs(res - np.linalg.norm(M @ w - y)) <= 1e-12 * res

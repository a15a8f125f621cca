"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test targets a plausible mistake: a wrong sign or factor in the drift of
Eq. convection, a wrong Neel constant (Sec. 2.1), a wrong basis convention,
quadrature or integrator error.  No test compares the oracle with itself.
"""
import numpy as np
import pytest
import scipy.special as ss

from oracle import equilibrium, galerkin, legendre1d, physics, radau, solve, sphere

MAT = physics.Material()


def null_state(A):
    """Stationary Galerkin state with c00 = 1/sqrt(4 pi) (row 0 of A is zero)."""
    c = np.zeros(A.shape[0])
    c[0] = 1.0 / np.sqrt(4 * np.pi)
    c[1:] = np.linalg.solve(A[1:, 1:], -A[1:, 0] * c[0])
    return c


# ------------------------------------------------------------ basis -------
def test_real_sh_matches_scipy_library():
    """Real SH = library complex SH with the CS phase removed (textbook)."""
    rng = np.random.default_rng(1)
    th, ph = rng.uniform(0.05, np.pi - 0.05, 7), rng.uniform(0, 2 * np.pi, 7)
    Y = sphere.real_sh(6, th, ph)
    for l in range(7):
        for m in range(-l, l + 1):
            yc = ss.sph_harm_y(l, abs(m), th, ph)
            ref = yc.real if m == 0 else np.sqrt(2) * (-1) ** abs(m) * (yc.real if m > 0 else yc.imag)
            np.testing.assert_allclose(Y[sphere.idx(l, m)], ref, atol=1e-13)


def test_real_sh_orthonormal_and_l1_is_cartesian():
    T, P, W, pts = sphere.quadrature(12, 24)
    Y = sphere.real_sh(8, T, P)
    np.testing.assert_allclose((Y * W) @ Y.T, np.eye(81), atol=1e-13)
    s = np.sqrt(3 / (4 * np.pi))
    np.testing.assert_allclose(Y[sphere.idx(1, 1)], s * pts[:, 0], atol=1e-14)
    np.testing.assert_allclose(Y[sphere.idx(1, -1)], s * pts[:, 1], atol=1e-14)
    np.testing.assert_allclose(Y[sphere.idx(1, 0)], s * pts[:, 2], atol=1e-14)


def test_tangential_gradient_central_difference():
    rng = np.random.default_rng(2)
    th, ph = rng.uniform(0.3, 2.8, 5), rng.uniform(0, 6.2, 5)
    Y, G = sphere.real_sh_with_grad(7, th, ph)
    h = 1e-6
    Yt = (sphere.real_sh(7, th + h, ph) - sphere.real_sh(7, th - h, ph)) / (2 * h)
    Yp = (sphere.real_sh(7, th, ph + h) - sphere.real_sh(7, th, ph - h)) / (2 * h)
    e_t = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], -1)
    e_p = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], -1)
    ref = Yt[..., None] * e_t + (Yp / np.sin(th))[..., None] * e_p
    np.testing.assert_allclose(G, ref, atol=2e-8)


# ------------------------------------------------------------ operator ----
def test_conservation_row_zero():
    """Mass conservation (Sec. 2.1, conservative discretisation): row 0 of A is 0."""
    P = physics.derive(MAT, 5e3, 22e-9)
    A0, A1 = galerkin.weak_form_matrices(8, P, physics.easy_axis(1.0, 2.0))
    scale = max(np.abs(A0).max(), np.abs(A1).max())
    assert np.abs(A0[0]).max() <= 1e-15 * scale
    assert np.abs(A1[:, 0]).max() <= 1e-15 * scale


def test_laplacian_eigenvalues_give_tau():
    """Free rotational diffusion: Y_l decays at rate l(l+1)/(2 tau) (Sec. 2.1, tau)."""
    P = physics.derive(MAT, 0.0, 20e-9)
    A0, _ = galerkin.weak_form_matrices(6, P, np.array([0, 0, 1.0]))
    lam = np.array([l * (l + 1) for l in range(7) for _ in range(2 * l + 1)])
    np.testing.assert_allclose(np.diag(A0), -lam / (2 * P.tau), rtol=1e-13)
    np.testing.assert_allclose(A0 - np.diag(np.diag(A0)), 0, atol=1e-12 * abs(A0).max())
    # tau value from the Sec. 2.1 formula, independently restated
    V = np.pi * 20e-9 ** 3 / 6
    gt = 1.76e11 / 1.01
    assert P.tau == pytest.approx(V * 474e3 / (2 * physics.K_BOLTZMANN * 293 * gt * 0.1), rel=1e-14)


@pytest.mark.parametrize("xi", [0.5, 3.0, 6.0])
def test_langevin_limit(xi):
    """K = 0, static field: stationary <m> = L(xi) H/|H| (Eq. Langevin), with
    geometric convergence in the truncation degree."""
    P = physics.derive(MAT, 0.0, 20e-9)
    Bdir = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    B = xi / P.bT * Bdir
    errs = []
    for L in (8, 14, 22):
        A0, A1 = galerkin.weak_form_matrices(L, P, np.array([0, 0, 1.0]))
        c = null_state(A0 + np.einsum("k,kij->ij", B, A1))
        errs.append(np.abs(galerkin.mean_moment(c) - equilibrium.langevin(xi) * Bdir).max())
    assert errs[-1] < 1e-12
    assert errs[0] > errs[1] > errs[2] or errs[1] < 1e-13


def test_boltzmann_with_anisotropy_is_stationary():
    """Static field, tilted easy axis: the Galerkin stationary state equals
    brute-force quadrature of exp(beta H.m + sigma (n.m)^2).  This holds only if
    2 sigma p1 = beta p3 and the signs of all four drift terms are right."""
    P = physics.derive(MAT, 4e3, 21e-9)
    n = physics.easy_axis(1.1, 0.7)
    B = np.array([0.004, -0.006, 0.003])
    A0, A1 = galerkin.weak_form_matrices(22, P, n)
    c = null_state(A0 + np.einsum("k,kij->ij", B, A1))
    mean, _ = equilibrium.boltzmann_mean(P.bT, B, P.sigma, n)
    np.testing.assert_allclose(galerkin.mean_moment(c), mean, atol=1e-12)
    # the projected Boltzmann density is the same state up to truncation, which
    # only touches the highest degrees
    np.testing.assert_allclose(galerkin.boltzmann_coeffs(22, P, n, B)[:81], c[:81], atol=1e-12)


def test_larmor_precession_sense_and_rate():
    """LLG precession: d<m>/dt has the component gamma~ B x <m> (Sec. 2.1,
    p1 = gamma~ mu0), positive sense about B.  State symmetric about x, B along z:
    the y-rate equals gamma~ Bz <m_x> exactly (damping and diffusion give no y part)."""
    P = physics.derive(MAT, 0.0, 20e-9)
    c = galerkin.boltzmann_coeffs(10, P, np.array([0, 0, 1.0]), np.array([0.01, 0, 0]))
    _, A1 = galerkin.weak_form_matrices(10, P, np.array([0, 0, 1.0]))
    Bz = 0.02
    rate = galerkin.mean_moment(Bz * A1[2] @ c)
    mx = galerkin.mean_moment(c)[0]
    assert rate[1] == pytest.approx(P.gt * Bz * mx, rel=1e-12)
    assert rate[1] > 0


def test_neel_small_barrier_slope_and_1d_solver():
    """H = 0: the slowest rate of <n.m> is (1/tau)(1 - 2 sigma/5 + O(sigma^2))
    (first-order perturbation of the m = 0 Legendre operator), and it equals the
    exact eigenvalue of the independent 1-D Legendre solver."""
    for K in (20.0, 200.0):
        P = physics.derive(MAT, K, 20e-9)
        A0, _ = galerkin.weak_form_matrices(12, P, np.array([0, 0, 1.0]))
        ev = np.sort(np.linalg.eigvals(A0).real)
        lam3d = -ev[-2]
        G = legendre1d.galerkin_1d(12, P.D, lambda x: 2 * P.sigma * x)
        lam1d = -np.sort(np.linalg.eigvals(G).real)[-2]
        assert lam3d == pytest.approx(lam1d, rel=1e-11)
        slope = (lam3d * P.tau - 1) / P.sigma
        assert slope == pytest.approx(-0.4, abs=0.6 * P.sigma)


def test_neel_high_barrier_brown_asymptote():
    """sigma >> 1: tau_N ~ tau (sqrt(pi)/2) sigma^{-3/2} e^sigma (Brown)."""
    P = physics.derive(MAT, 1.5e4, 20e-9)           # sigma ~ 15.5
    G = legendre1d.galerkin_1d(60, P.D, lambda x: 2 * P.sigma * x)
    lam = -np.sort(np.linalg.eigvals(G).real)[-2]
    brown = P.tau * np.sqrt(np.pi) / 2 * P.sigma ** -1.5 * np.exp(P.sigma)
    assert 1.0 / lam == pytest.approx(brown, rel=0.1)


def test_rotation_covariance():
    """Rotating field and easy axis together rotates the mean moment."""
    P = physics.derive(MAT, 3e3, 20e-9)
    n = physics.easy_axis(0.4, 0.3)
    B = np.array([0.006, 0.002, -0.004])
    a, b = 0.9, -1.3
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    R = Rz @ Rx
    ms = []
    for nn, BB in ((n, B), (R @ n, R @ B)):
        A0, A1 = galerkin.weak_form_matrices(10, P, nn)
        A = A0 + np.einsum("k,kij->ij", BB, A1)
        c0 = galerkin.boltzmann_coeffs(10, P, nn, np.zeros(3))
        # short trajectory from the zero-field state into the field
        from scipy.linalg import expm
        ms.append(galerkin.mean_moment(expm(A * 2e-8) @ c0))
    np.testing.assert_allclose(R @ ms[0], ms[1], atol=1e-12)


# ------------------------------------------------------------ integrator --
def test_radau_tableau_order_conditions():
    a, b, c = radau.radau_iia_tableau(3)
    np.testing.assert_allclose(c, [(4 - np.sqrt(6)) / 10, (4 + np.sqrt(6)) / 10, 1.0], atol=1e-15)
    for q in range(1, 6):                      # quadrature order 2s - 1 = 5
        assert np.dot(b, c ** (q - 1)) == pytest.approx(1.0 / q, abs=1e-14)
    for q in range(1, 4):                      # stage order 3: C(3)
        np.testing.assert_allclose(a @ c ** (q - 1), c ** q / q, atol=1e-14)


def test_radau_converges_on_time_dependent_scalar():
    """y' = (-1 + 5 cos t) y, y(0)=1 has y = exp(-t + 5 sin t); fixed steps show order 5."""
    f = lambda t: np.array([[-1 + 5 * np.cos(t)]])
    errs = []
    for nstep in (20, 40):
        integ = radau.RadauIIA(f, rtol=1.0, atol=1e300)        # error control off
        t, y = 0.0, np.array([1.0])
        h = 3.0 / nstep
        for _ in range(nstep):
            y = integ.step(t, y, h)
            t += h
        errs.append(abs(y[0] - np.exp(-3.0 + 5 * np.sin(3.0))))
    assert np.log2(errs[0] / errs[1]) > 4.7


def test_free_diffusion_trajectory():
    """Field switched off after a Boltzmann start: <m>(t) = <m>(0) exp(-t/tau)."""
    P = physics.derive(MAT, 0.0, 20e-9)
    drv = physics.Drive(amp=(0, 0, 0), freq=(1e6, 1e6, 1e6), phase=(0, 0, 0), period=1e-7)
    inst = solve.Instance(h_off=(0, 0, 0), theta=0.3, phi=0.2, K=0.0, d=20e-9, L=6)
    r = solve.solve_instance(MAT, drv, inst, solve.Schedule(20, 0, 1), rtol=1e-11,
                             ic_field=np.array([0.004, 0.002, -0.003]))
    ref = r["m"][0] * np.exp(-r["t"] / P.tau)[:, None]
    np.testing.assert_allclose(r["m"], ref, atol=1e-12)
    np.testing.assert_allclose(r["dmdt"], -ref / P.tau, rtol=1e-9, atol=1e-6)


def test_axial_field_matches_1d_solver():
    """K = 0, field along x only: <m_y> = <m_z> = 0 and <m_x>(t) equals the 1-D
    Legendre solve of the same drive."""
    f = 25e3
    drv = physics.Drive(amp=(0.012, 0, 0), freq=(f, f, f), phase=(0.3, 0, 0), period=1 / f)
    inst = solve.Instance(h_off=(0.002, 0, 0), theta=0.0, phi=0.0, K=0.0, d=20e-9, L=12)
    sched = solve.Schedule(40, 0, 1)
    r = solve.solve_instance(MAT, drv, inst, sched, rtol=1e-11)
    assert np.abs(r["m"][:, 1:]).max() < 1e-14
    P = physics.derive(MAT, 0.0, 20e-9)
    G1 = legendre1d.galerkin_1d(12, P.D, lambda x: P.bT + 0 * x)   # U = bT B x, unit field
    G0 = legendre1d.galerkin_1d(12, P.D, lambda x: 0 * x)
    A_of_t = lambda t: G0 + drv.field(t, (0.002, 0, 0))[0] * (G1 - G0)
    c0 = legendre1d.equilibrium(12, lambda x: P.bT * drv.field(0.0, (0.002, 0, 0))[0] * x)
    integ = radau.RadauIIA(A_of_t, rtol=1e-12, h0=1e-10, h_max=drv.period / 40)
    C = integ.integrate(0.0, c0, solve.sample_times(drv, sched))
    np.testing.assert_allclose(r["m"][:, 0], legendre1d.mean_x(C), atol=1e-10)


def test_halfwave_symmetry_of_sinusoidal_drive():
    """B(t + T/2) = -B(t) with n in the x-y plane: after the transient,
    <m>(t + T/2) = (-m_x, -m_y, m_z)(t) (rotation by pi about z maps n to -n,
    an equivalent axis), so m_x, m_y carry odd harmonics only."""
    f = 25e3
    drv = physics.Drive(amp=(0.012, 0, 0), freq=(f, f, f), phase=(0, 0, 0), period=1 / f)
    inst = solve.Instance(h_off=(0, 0, 0), theta=np.pi / 2, phi=np.pi / 4, K=2e3, d=20e-9, L=6)
    r = solve.solve_instance(MAT, drv, inst, solve.Schedule(100, 1, 1), rtol=1e-10)
    m = r["m"]
    np.testing.assert_allclose(m[50:, :2], -m[:50, :2], atol=1e-9)
    np.testing.assert_allclose(m[50:, 2], m[:50, 2], atol=1e-9)


def test_self_convergence_in_rtol():
    f = 25e3
    drv = physics.Drive(amp=(0.012, 0, 0), freq=(f, f, f), phase=(0, 0, 0), period=1 / f)
    inst = solve.Instance(h_off=(0.001, 0.002, 0), theta=1.2, phi=0.5, K=3e3, d=19e-9, L=8)
    sched = solve.Schedule(50, 0, 1)
    a = solve.solve_instance(MAT, drv, inst, sched, rtol=1e-10)["m"]
    b = solve.solve_instance(MAT, drv, inst, sched, rtol=1e-11)["m"]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10


# ------------------------------------------------------------ signal ------
def test_phi_hat_matches_fft_and_single_tone():
    rng = np.random.default_rng(3)
    S = 96
    d = rng.normal(size=(S, 3))
    ch = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    ph = solve.phi_hat(d, ch, S, 40)
    np.testing.assert_allclose(ph[0], np.fft.fft(d[:, 0])[:41] / S, atol=1e-14)
    np.testing.assert_allclose(ph[1], np.fft.fft(d[:, 1])[:41] / S, atol=1e-14)
    j = np.arange(S)
    tone = np.stack([np.cos(2 * np.pi * 5 * j / S), np.zeros(S), np.zeros(S)], 1)
    p = solve.phi_hat(tone, ch[:1], S, 10)[0]
    assert abs(p[5] - 0.5) < 1e-14 and np.abs(np.delete(p, 5)).max() < 1e-14

"""Adjoint-driven fit (paper_2106_08040_gb300/fit.py): the misfit gradient of a
candidate parameter set, summed over a voxel grid through fp_grad, against
central differences of the misfit itself (relative step 1e-4, forward at
rtol 1e-11; agreement 1e-4 of the gradient norm), and a descent step along it
lowers the misfit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_08040_gb300 import build, workloads      # noqa: E402

pytestmark = pytest.mark.gpu

DSPEC = workloads.DriveSpec(amp=(0.010, 0.008, 0.0), freq=(50e3, 75e3, 0.0), phase=(0.0, 0.0, 0.0),
                            period=4e-5, samples_per_period=64, warmup_periods=0, output_periods=1)


@pytest.fixture(scope="module")
def problem():
    build.build()
    from paper_2106_08040_gb300 import fit
    offs = workloads.voxel_offsets(4, 4, fov=8e-3)
    pb = fit.FitProblem(DSPEC, offs, L=8, k_max=20, rtol=1e-11)
    hidden = np.array([[1.5e3, 19e-9, np.pi / 2, 0.3], [2.5e3, 21e-9, 1.2, 1.1]])
    u = pb.measurement(hidden, [0.6, 0.4], noise=0.01, seed=3)
    yield pb, u
    pb.close()


def test_misfit_gradient_matches_central_differences(problem):
    pb, u = problem
    cand = np.array([[1.2e3, 20e-9, 1.4, 0.5], [2.0e3, 18e-9, 1.0, 0.9]])
    J, g, ok = pb.misfit_and_grad(cand, u)
    assert ok
    fd = np.zeros_like(g)
    for j in range(4):
        step = 1e-4 * np.abs(cand[:, j]) if j < 2 else np.full(len(cand), 1e-4)
        a, b = cand.copy(), cand.copy()
        a[:, j] += step
        b[:, j] -= step
        Ja, _, _ = pb.misfit_and_grad(a, u)
        Jb, _, _ = pb.misfit_and_grad(b, u)
        fd[:, j] = (Ja - Jb) / (2 * step)
    w = np.array([cand[0, 0], cand[0, 1], 1.0, 1.0])
    for c in range(len(cand)):
        scale = np.linalg.norm(fd[c] * w)
        assert np.abs((g[c] - fd[c]) * w).max() <= 1e-4 * scale, (c, g[c], fd[c])


def test_descent_step_lowers_the_misfit(problem):
    pb, u = problem
    p = np.array([[1.2e3, 20e-9, 1.4, 0.5]])
    J0, g, ok = pb.misfit_and_grad(p, u)
    assert ok
    w = np.array([p[0, 0], p[0, 1], 1.0, 1.0])           # step in relative units for K and d
    d = -(g[0] * w) / np.linalg.norm(g[0] * w)
    p1 = p + 0.01 * d * w
    J1, _, _ = pb.misfit_and_grad(p1, u)
    assert J1[0] < J0[0]


def test_adam_fit_recovers_a_single_hidden_set(problem):
    """Noise-free measurement of one hidden set; starting 15 % off in K and d
    and 0.15 rad off in both angles, twelve adjoint-driven Adam steps lower
    the misfit by more than a factor of 4."""
    pb, _ = problem
    hidden = np.array([[1.6e3, 20e-9, 1.3, 0.7]])
    u = pb.measurement(hidden, [1.0], noise=0.0)
    start = hidden * np.array([[1.15, 0.85, 1.0, 1.0]]) + np.array([[0.0, 0.0, 0.15, -0.15]])
    p, hist = pb.fit(start, u, iters=12, lr=0.03)
    assert hist[-1][0] < 0.25 * hist[0][0], hist[:, 0]


def test_superposition_gradients_match_central_differences(problem):
    """Superposition model sum_j w_j phi_hat(p_j): dJ/dw_j against central
    differences of J in w_j, dJ/dp_j against central differences in p_j
    (relative step 1e-4, forward at rtol 1e-11; agreement 1e-4 of the norm)."""
    pb, u = problem
    cand = np.array([[1.4e3, 19.5e-9, 1.5, 0.4], [2.2e3, 20.5e-9, 1.1, 1.0]])
    w = np.array([0.55, 0.5])
    J, g, gw, ok = pb.superposition_misfit_and_grad(cand, w, u)
    assert ok
    fdw = np.zeros(2)
    for j in range(2):
        a, b = w.copy(), w.copy()
        a[j] += 1e-4
        b[j] -= 1e-4
        fdw[j] = (pb.superposition_misfit_and_grad(cand, a, u)[0] - pb.superposition_misfit_and_grad(cand, b, u)[0]) / 2e-4
    assert np.abs(gw - fdw).max() <= 1e-6 * np.linalg.norm(fdw), (gw, fdw)
    for j in range(2):
        fd = np.zeros(4)
        for k in range(4):
            step = 1e-4 * abs(cand[j, k]) if k < 2 else 1e-4
            a, b = cand.copy(), cand.copy()
            a[j, k] += step
            b[j, k] -= step
            fd[k] = (pb.superposition_misfit_and_grad(a, w, u)[0] - pb.superposition_misfit_and_grad(b, w, u)[0]) / (2 * step)
        sc = np.array([cand[j, 0], cand[j, 1], 1.0, 1.0])
        assert np.abs((g[j] - fd) * sc).max() <= 1e-4 * np.linalg.norm(fd * sc), (j, g[j], fd)


def test_superposition_fit_recovers_two_hidden_sets_with_weights(problem):
    """Two hidden sets with weights 0.6 / 0.4 (1 % noise); starting 10 % off in
    K and d, 0.1 rad off in the angles and at equal weights 0.5 / 0.5, adjoint-
    driven Adam on the parameters and weights lowers the misfit by more than a
    factor of 10 and moves both weights towards their hidden values."""
    pb, u = problem
    hidden = np.array([[1.5e3, 19e-9, np.pi / 2, 0.3], [2.5e3, 21e-9, 1.2, 1.1]])
    start = hidden * np.array([[1.1, 0.9, 1.0, 1.0], [0.9, 1.1, 1.0, 1.0]]) + np.array([[0, 0, -0.1, 0.1], [0, 0, 0.1, -0.1]])
    p, w, hist = pb.fit_superposition(start, [0.5, 0.5], u, iters=25, lr=0.03)
    assert hist[-1] < 0.1 * hist[0], hist
    assert abs(w[0] - 0.6) < abs(0.5 - 0.6) and abs(w[1] - 0.4) < abs(0.5 - 0.4), w

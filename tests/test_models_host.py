"""Host-side entry points of the Sec. 2.3 distance measures (no GPU): the
mixing orders of Eq. mix and the frequency index set I_freq, bit-exact against
the oracle."""
import numpy as np
import pytest

from oracle import models


@pytest.fixture(scope="module")
def fp():
    from paper_2106_08040_gb300 import build
    build.build()
    from paper_2106_08040_gb300 import fp as fpmod
    return fpmod


@pytest.mark.parametrize("n_dens", [16, 5, 1])
def test_mixing_order_matches_oracle(fp, n_dens):
    for k in list(range(0, 817)) + [-1, -17, -400, 5000]:
        assert fp.fp_mixing_order(k, n_dens) == models.mixing_order(k, n_dens), k


def test_freq_index_set_matches_oracle(fp):
    for mx, my in ((3, 2), (20, 20), (0, 5), (1, 1)):
        ref = models.freq_index_set(mx, my, 16)
        ref = ref[ref <= 816]
        np.testing.assert_array_equal(fp.fp_freq_index_set(mx, my, 16, 816), ref)


def _rand_complex(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _gram(M, y):
    My = np.concatenate([M, y[:, None]], axis=1)
    G = np.conj(My.T) @ My
    return np.ascontiguousarray(np.stack([G.real, G.imag], -1))


def test_m2_solve_recovers_planted_weights(fp):
    """Host M2 solve (fp_m2_solve) from an exact Gram matrix: a planted
    non-negative superposition is recovered with zero residual."""
    rng = np.random.default_rng(5)
    Psi = [[_rand_complex(rng, (40, 2, 12)) for _ in range(6)] for _ in range(3)]
    w_true = np.array([0.0, 1.5, 0.0, 0.25, 2.0, 0.0])
    S = [sum(w * p for w, p in zip(w_true, Pa)) for Pa in Psi]
    ks = np.arange(1, 12)
    M, y = models.m2_matrix(Psi, S, ks)
    w, obj, res, sv, s = fp.fp_m2_solve(_gram(M, y), 6)
    assert s == 6
    np.testing.assert_allclose(w, w_true, atol=1e-8)
    assert res <= 1e-12 * np.vdot(y, y).real
    np.testing.assert_allclose(sv, np.linalg.svd(M, compute_uv=False), rtol=1e-10)


@pytest.mark.parametrize("s_rank", [0, 4])
def test_m2_solve_matches_oracle(fp, s_rank):
    """Noisy data: full rank (unique minimiser: the weights agree) and a
    truncated SVD of rank 4 < J = 6 (the minimiser is not unique; the
    truncated objective, which is, agrees, and the weights are feasible)."""
    rng = np.random.default_rng(6)
    Psi = [[_rand_complex(rng, (40, 2, 12)) for _ in range(6)] for _ in range(3)]
    S = [sum(w * p for w, p in zip([1.0, 0.5, 0.0, 2.0, 0.1, 0.0], Pa)) + 0.3 * _rand_complex(rng, (40, 2, 12))
         for Pa in Psi]
    ks = np.arange(12)
    M, y = models.m2_matrix(Psi, S, ks)
    w, obj, res, sv, s = fp.fp_m2_solve(_gram(M, y), 6, s_rank)
    wo, reso, svo, objo = models.m2_weights(Psi, S, ks, s_rank=s_rank or None)
    assert (w >= 0).all()
    if s_rank == 0:
        np.testing.assert_allclose(w, wo, atol=1e-7 * np.abs(wo).max())
        assert abs(np.sqrt(res) - reso) <= 1e-9 * reso
    else:
        assert s == 4
        assert abs(obj - objo) <= 1e-9 * objo
        assert abs(np.sqrt(res) - np.linalg.norm(M @ w - y)) <= 1e-9 * np.linalg.norm(y)


def test_m2_solve_degenerate_problems(fp):
    """Degenerate M2 problems with a unique answer: zero data gives zero
    weights; data in the negative cone of the dictionary gives zero weights; a
    dictionary column that is identically zero gets weight 0 while the others
    equal a library NNLS solve of the real-split least-squares problem; an
    all-zero dictionary has rank 0 and zero weights."""
    scipy_optimize = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(11)
    M = _rand_complex(rng, (50, 4))
    w, obj, res, sv, s = fp.fp_m2_solve(_gram(M, np.zeros(50, complex)), 4)
    assert s == 4 and (w == 0).all() and res == 0.0
    w, _, _, _, _ = fp.fp_m2_solve(_gram(M, -(M @ np.array([1.0, 0.5, 0.2, 0.3]))), 4)
    assert (w == 0).all()
    y = M @ np.array([1.0, 0.5, 0.2, 0.3]) + 0.1 * _rand_complex(rng, 50)
    Mz = M.copy()
    Mz[:, 2] = 0.0
    w, obj, res, sv, s = fp.fp_m2_solve(_gram(Mz, y), 4)
    ref, rnorm = scipy_optimize.nnls(np.concatenate([Mz.real, Mz.imag]), np.concatenate([y.real, y.imag]))
    assert s == 3 and w[2] == 0.0 and sv[3] == 0.0
    np.testing.assert_allclose(w, ref, rtol=1e-9, atol=1e-12)
    assert abs(res - rnorm ** 2) <= 1e-9 * rnorm ** 2
    w, obj, res, sv, s = fp.fp_m2_solve(_gram(np.zeros((10, 3), complex), np.zeros(10, complex)), 3)
    assert s == 0 and (w == 0).all() and (sv == 0).all()

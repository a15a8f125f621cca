"""GPU parity of the Sec. 2.2 models M0 and M1 and of the Sec. 2.3 measures
(libfp.so through its C ABI) against the FP64 oracle (oracle/models.py).

Bars.  M0 is a closed form evaluated in FP64 on both sides (the GPU by the
analytic chain rule, the oracle by the complex-step derivative): each output
is a few dozen rounded operations on O(1) quantities, and the Langevin
function and its derivative are conditioned at most ~ 1/x^2 ~ 4 where the
series takes over (x = 0.5), so the relative L2 bar is 1e-13 on m and 1e-12
on d<m>/dt (whose terms cancel near a field zero crossing by up to ~10).  M1
and the NRMSE are sums of N products (relative rounding ~ N eps ~ 1e-13 for
N ~ 1000): bar 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_08040_gb300 import build, workloads      # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    build.build()
    from paper_2106_08040_gb300 import fp as fpmod
    return fpmod


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def test_m0_traces_and_phi_hat_match_oracle(fp):
    from oracle import models, physics, solve
    dspec, inst = workloads.system_matrix_workload()
    # voxels: grid corner, one next to the centre (field zero crossings), an edge, and a d <= 0 record
    pick = [0, 16 * 32 + 15, 16 * 32 + 16, 31 * 32 + 5, 7]
    sub = inst[pick].copy()
    sub["d"][1] = 14e-9
    sub["d"][4] = 0.0
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(), 8)
    n, S = len(sub), ctx.num_samples()
    d_inst = fp.instances_to_device(sub, "cuda")
    m = torch.empty((n, S, 3), dtype=torch.float64, device="cuda")
    dm = torch.empty_like(m)
    fp.fp_equilibrium(ctx, d_inst, n, m, dm)
    ph = torch.empty((n, 2, 817, 2), dtype=torch.float64, device="cuda")
    ch = [[1.0, 0, 0], [0, 1.0, 0]]
    fp.fp_signal(ctx, dm, n, 816, ch, ph)
    torch.cuda.synchronize()
    drv = physics.Drive(amp=dspec.amp, freq=dspec.freq, phase=dspec.phase, period=dspec.period)
    t = solve.sample_times(drv, solve.Schedule(dspec.samples_per_period, dspec.warmup_periods, dspec.output_periods))
    mm, dd, pp = m.cpu().numpy(), dm.cpu().numpy(), ph.cpu().numpy()
    for i in range(n - 1):
        mo, do = models.equilibrium_trace(physics.Material(), drv, float(sub["d"][i]), sub["h_off"][i], t)
        assert rel(mm[i], mo) <= 1e-13, i
        assert rel(dd[i], do) <= 1e-12, i
        po = solve.phi_hat(do, ch, dspec.samples_per_period, 816)
        assert rel(pp[i, ..., 0] + 1j * pp[i, ..., 1], po) <= 1e-12, i
    assert float(m[n - 1].abs().max()) == 0.0 and float(dm[n - 1].abs().max()) == 0.0


def _cplx(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _dev(z):
    return torch.from_numpy(np.ascontiguousarray(np.stack([z.real, z.imag], -1))).cuda()


@pytest.mark.parametrize("N,C,K1,Q", [(1021, 2, 817, 3), (5, 1, 3, 1), (64, 2, 64, 2)])
def test_m1_fit_matches_oracle(fp, N, C, K1, Q):
    """Several column blocks with a ragged tail (C K1 not a multiple of 64) and
    a voxel count not a multiple of the voxel groups; one element fits
    exactly (planted filter), one row of Phi is zero."""
    from oracle import models
    rng = np.random.default_rng(N + Q)
    Phi = _cplx(rng, (Q, N, C, K1))
    a_true = _cplx(rng, (C, K1))
    S = a_true[None] * Phi[0] + (0.05 * _cplx(rng, (N, C, K1)) if Q > 1 else 0.0)
    if Q > 1:
        Phi[1, :, 0, 1] = 0.0
    d_phi, d_S = _dev(Phi), _dev(S)
    a = torch.empty((Q, C, K1, 2), dtype=torch.float64, device="cuda")
    eps = torch.empty((Q, C, K1), dtype=torch.float64, device="cuda")
    smax = torch.empty((C, K1), dtype=torch.float64, device="cuda")
    fp.fp_m1_fit(d_phi, Q, d_S, N, C, K1, a, eps, smax)
    torch.cuda.synchronize()
    ag = a.cpu().numpy()
    ag = ag[..., 0] + 1j * ag[..., 1]
    eg = eps.cpu().numpy()
    for q in range(Q):
        ao, eo = models.m1_fit(Phi[q], S)
        ok = np.isfinite(ao)
        assert rel(ag[q][ok], ao[ok]) <= 1e-12, q
        assert (ag[q][~ok] == 0).all()
        eo = np.where(ok, eo, np.sqrt(np.mean(np.abs(S) ** 2, 0)) / np.abs(S).max(0))
        # eps is relative to ||S_k||_inf: rounding of an exact fit leaves ~1e-16
        assert np.abs(eg[q] - eo).max() <= 1e-12 * np.abs(eo).max() + 1e-14, q
    np.testing.assert_allclose(smax.cpu().numpy(), np.abs(S).max(0), rtol=1e-15)
    if Q == 1:
        assert eg.max() <= 1e-13


def test_nrmse_matches_oracle(fp):
    from oracle import models
    rng = np.random.default_rng(9)
    A, C, K1 = 12, 2, 817
    eps = rng.uniform(0.05, 0.4, size=(A, C, K1))
    ks = fp.fp_freq_index_set(20, 20, 16, K1 - 1)
    d_eps = torch.from_numpy(eps).cuda()
    d_ks = torch.from_numpy(ks.astype(np.int32)).cuda()
    ef = torch.empty(K1, dtype=torch.float64, device="cuda")
    eg = torch.empty(1, dtype=torch.float64, device="cuda")
    fp.fp_nrmse(d_eps, A, C, K1, d_ks, len(ks), ef, eg)
    torch.cuda.synchronize()
    assert rel(ef.cpu().numpy(), models.eps_freq(eps)) <= 1e-14
    assert abs(float(eg.item()) - models.eps_global(eps, ks)) <= 1e-14 * models.eps_global(eps, ks)


def test_empty_inputs_are_noops(fp):
    dspec, inst = workloads.system_matrix_workload()
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(), 8)
    fp.fp_equilibrium(ctx, fp.instances_to_device(inst[:1], "cuda"), 0, None,
                      torch.empty(1, dtype=torch.float64, device="cuda"))
    z = torch.zeros(2, dtype=torch.float64, device="cuda")
    fp.fp_m1_fit(z, 0, z, 4, 1, 1, z, z, z)
    torch.cuda.synchronize()


@pytest.mark.parametrize("A,J,N,C,K1,nk", [(3, 6, 40, 2, 12, 11), (2, 37, 29, 2, 50, 23)])
def test_m2_gram_and_weights_match_oracle(fp, A, J, N, C, K1, nk):
    """fp_m2_gram against the oracle's explicit Sigma-weighted matrix [M | y]
    (sums of R = A N C nk products: bar 1e-12 relative to the largest entry),
    tiles with a ragged edge (J + 1 not a multiple of 16), a row subset ks;
    then the host M2 solve from the GPU Gram matrix against the oracle's
    weights (full rank: the minimiser is unique)."""
    from oracle import models
    rng = np.random.default_rng(A * 100 + J)
    Phi = _cplx(rng, (A, J, N, C, K1))
    a = _cplx(rng, (A, J, C, K1))
    w_true = np.abs(rng.normal(size=J)) * (rng.uniform(size=J) < 0.5)
    Psi = [[a[t, j][None] * Phi[t, j] for j in range(J)] for t in range(A)]
    S = [sum(w_true[j] * Psi[t][j] for j in range(J)) + 0.05 * _cplx(rng, (N, C, K1)) for t in range(A)]
    ks = np.sort(rng.choice(K1, size=nk, replace=False)).astype(np.int32)
    smax = np.stack([np.abs(St).max(0) for St in S])
    G = torch.empty((J + 1, J + 1, 2), dtype=torch.float64, device="cuda")
    fp.fp_m2_gram(_dev(Phi), _dev(a), _dev(np.stack(S)), torch.from_numpy(smax).cuda(), A, J, N, C, K1,
                  torch.from_numpy(ks).cuda(), nk, G)
    torch.cuda.synchronize()
    Gg = G.cpu().numpy()
    Gg = Gg[..., 0] + 1j * Gg[..., 1]
    M, y = models.m2_matrix(Psi, S, ks)
    My = np.concatenate([M, y[:, None]], axis=1)
    Go = np.conj(My.T) @ My
    iu = np.triu_indices(J + 1)
    assert np.abs(Gg[iu] - Go[iu]).max() <= 1e-12 * np.abs(Go).max()
    Gfull = np.triu(Gg) + np.conj(np.triu(Gg, 1).T)
    w, obj, res, sv, s = fp.fp_m2_solve(np.stack([Gfull.real, Gfull.imag], -1), J)
    wo, reso, svo, objo = models.m2_weights(Psi, S, ks)
    assert s == J
    np.testing.assert_allclose(w, wo, atol=1e-7 * np.abs(wo).max())
    assert abs(np.sqrt(res) - reso) <= 1e-8 * reso

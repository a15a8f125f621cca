"""GPU parity of the CUDA path (libfp.so through its C ABI) against the FP64 oracle.

Trace bar: relative L2 error of the magnetization trace <= 1e-9
(||m_gpu - m_oracle||_2 / ||m_oracle||_2 over all samples and components, per
instance).

Derivative bar, derived (not fitted): d<m>/dt = sqrt(4 pi/3) (A(t_j) c)_{l=1}
takes the difference of large terms, so a state error dc costs |A_{l=1}| |dc|
in d<m>/dt while the trace sees only dc_{l=1}.  The integrator keeps the local
state error of every step below rtol max|c| (max norm) and the operator damps
every non-conserved mode within a sample interval (relaxation time ~ 26 ns
against a 400 ns spacing at sigma = 2), so the state error at a sample is at
most the sum of the local errors of the steps inside the last sample
interval: G rtol max|c| with G = ceil(accepted steps / samples) from the
kernel's own counters over the (warm-up + output) sample intervals (2 for
5 stages, 5 for 3 stages on the Lissajous workload).  How integration errors of the state map into d<m>/dt is measured
on the oracle alone: its self-convergence between rtol 1e-11 and 1e-12 gives
the state change eps_c (relative to max|c|) and the d<m>/dt change eps_d,
an amplification A = eps_d / eps_c.  The bar for a GPU run at rtol r is
    DTOL(r) = A G r + eps_d,
the second term bounding the oracle reference's own d<m>/dt error.  phi_hat,
a linear map of the last period's d<m>/dt, takes the same form with its own
eps_phi.  The goldens (tests/golden, oracle at rtol 1e-12) store eps_c,
eps_d and eps_phi; small on-the-fly cases compute them from two oracle solves.
"""
import glob
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_08040_gb300 import build, workloads      # noqa: E402

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")
TOL = 1e-9          # magnetization trace


def dtol(ref, rtol, key="selfconv_dmdt", G=1.0):
    """Derived bar DTOL(rtol) = (eps_key / eps_c) G rtol + eps_key of an oracle reference."""
    return float(ref[key]) / float(ref["selfconv_c"]) * G * rtol + float(ref[key])


def steps_per_interval(stats, dspec, rows=None):
    """G = ceil(accepted steps / sample intervals integrated), the largest over the
    given instances ((warm-up + output periods) x samples per period intervals)."""
    st = np.asarray(stats.cpu().numpy() if hasattr(stats, "cpu") else stats)
    if rows is not None:
        st = st[rows]
    intervals = (dspec.warmup_periods + dspec.output_periods) * dspec.samples_per_period
    return float(np.ceil(st[:, 0].max() / intervals))


@pytest.fixture(scope="module")
def fp():
    build.build()
    from paper_2106_08040_gb300 import fp as fpmod
    return fpmod


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def oracle_solve(dspec, rec, rtol=1e-11):
    from oracle import physics, solve
    drive = physics.Drive(amp=dspec.amp, freq=dspec.freq, phase=dspec.phase, period=dspec.period)
    sched = solve.Schedule(dspec.samples_per_period, dspec.warmup_periods, dspec.output_periods)
    inst = solve.Instance(h_off=tuple(rec["h_off"]), theta=float(rec["theta"]), phi=float(rec["phi"]),
                          K=float(rec["K"]), d=float(rec["d"]), L=int(rec["L"]))
    return solve.solve_instance(physics.Material(), drive, inst, sched, rtol=rtol, return_state=True)


def oracle_reference(dspec, rec, rtol=1e-12, rtol_check=1e-11):
    """Oracle solution at rtol with the self-convergence figures of the derived
    bar (a second solve at rtol_check)."""
    r12 = oracle_solve(dspec, rec, rtol)
    r11 = oracle_solve(dspec, rec, rtol_check)
    r12["selfconv_c"] = np.abs(r11["c"] - r12["c"]).max() / np.abs(r12["c"]).max()
    r12["selfconv_dmdt"] = rel(r11["dmdt"], r12["dmdt"])
    return r12


@pytest.mark.parametrize("stages", [3, 5])
def test_single_instance_trace(fp, stages):
    path = os.path.join(GOLD, "single_instance_L10.npz")
    if not os.path.exists(path):
        pytest.skip("golden trace not generated")
    ref = np.load(path)
    dspec, inst = workloads.single_instance_workload()
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-9, stages=stages), 10)
    m, dm, st, stats = fp.solve(ctx, inst)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    G = steps_per_interval(stats, dspec)
    assert rel(m.cpu().numpy()[0], ref["m"]) <= TOL
    assert rel(dm.cpu().numpy()[0], ref["dmdt"]) <= dtol(ref, 1e-9, G=G)


@pytest.mark.parametrize("stages", [3, 5])
def test_system_matrix_full_launch_sampled_voxels(fp, stages):
    """Full 32 x 32 batch in one launch (as the benchmark runs it, either
    Radau stage count); sampled voxels checked against oracle traces, every
    status OK."""
    files = sorted(glob.glob(os.path.join(GOLD, "sysmat_L16_v*.npz")))
    assert files, "no golden voxel traces"
    dspec, inst = workloads.system_matrix_workload()
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-9, stages=stages), 16)
    m, dm, st, stats = fp.solve(ctx, inst)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    mm, dd = m.cpu().numpy(), dm.cpu().numpy()
    for f in files:
        ref = np.load(f)
        k = int(ref["iy"]) * 32 + int(ref["ix"])
        G = steps_per_interval(stats, dspec, [k])
        assert rel(mm[k], ref["m"]) <= TOL, f
        assert rel(dd[k], ref["dmdt"]) <= dtol(ref, 1e-9, G=G), f
    # mirror symmetry (any size): with n || x, f_x T = 16, f_y T = 17 the field of
    # voxel (x, y) at t + T/2 is R_x(pi) applied to the field of voxel (x, -y) at t,
    # so m_(x,y)(t + T/2) = (m_x, -m_y, -m_z)_(x,-y)(t) in the periodic regime
    S = 1632
    for iy, ix in ((3, 5), (10, 16), (0, 31), (15, 0)):
        a = mm[iy * 32 + ix]
        b = mm[(31 - iy) * 32 + ix]
        shifted = np.roll(a, -S // 2, axis=0)
        mirrored = b * np.array([1.0, -1.0, -1.0])
        assert rel(shifted, mirrored) <= 10 * TOL


def test_ragged_degrees_random_instances(fp):
    """Uneven truncation degrees in one launch against the oracle (small sizes)."""
    dspec = workloads.DriveSpec(amp=(0.010, 0.004, 0.0), freq=(50e3, 50e3, 50e3), phase=(0.0, 0.7, 0.0),
                                period=2e-5, samples_per_period=64, warmup_periods=0, output_periods=1)
    inst = workloads.random_instances(5, 6, seed=7, max_offset=0.006)
    inst["L"] = [6, 8, 5, 6, 7]          # each resolves its instance (oracle |<m>| < 1)
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-10, stages=3), 8)
    m, dm, st, stats = fp.solve(ctx, inst)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    for i in range(len(inst)):
        r = oracle_reference(dspec, inst[i])
        G = steps_per_interval(stats, dspec, [i])
        assert rel(m.cpu().numpy()[i], r["m"]) <= TOL, i
        assert rel(dm.cpu().numpy()[i], r["dmdt"]) <= dtol(r, 1e-10, G=G), i


def test_unresolved_truncation_is_flagged(fp):
    """At L = 3 the truncated operator of this instance is not dissipative: the
    oracle's Galerkin solution at the same L reaches |<m>| = 1.39 > 1, and the
    solver must end it with FP_STATUS_UNRESOLVED (6) instead of returning it."""
    dspec = workloads.DriveSpec(amp=(0.010, 0.004, 0.0), freq=(50e3, 50e3, 50e3), phase=(0.0, 0.7, 0.0),
                                period=2e-5, samples_per_period=64, warmup_periods=0, output_periods=1)
    inst = workloads.random_instances(5, 6, seed=7, max_offset=0.006)[:1]
    inst["L"] = 3
    r = oracle_solve(dspec, inst[0], rtol=1e-8)
    assert np.linalg.norm(r["m"], axis=1).max() > 1.0
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-10, stages=3), 8)
    _, _, st, _ = fp.solve(ctx, inst)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == 6


def test_rotation_covariance(fp):
    """Rotating offset field and easy axis about the drive axis (z) rotates the
    whole trace <m>(t) (property at any size; exercises the easy-axis frame)."""
    dspec = workloads.DriveSpec(amp=(0.0, 0.0, 0.010), freq=(50e3, 50e3, 50e3), phase=(0.0, 0.0, 0.3),
                                period=2e-5, samples_per_period=100, warmup_periods=0, output_periods=1)
    a = 0.6
    R = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    n = np.array([np.sin(0.5) * np.cos(0.2), np.sin(0.5) * np.sin(0.2), np.cos(0.5)])
    off = np.array([0.002, -0.003, 0.001])
    inst = workloads.make_instances(2)
    inst["K"], inst["d"], inst["L"] = 3e3, 20e-9, 10
    for i, (nn, oo) in enumerate(((n, off), (R @ n, R @ off))):
        inst[i]["h_off"] = oo
        inst[i]["theta"], inst[i]["phi"] = np.arccos(nn[2]), np.arctan2(nn[1], nn[0])
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-10, stages=3), 10)
    m, dm, st, stats = fp.solve(ctx, inst)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    mm, dd = m.cpu().numpy(), dm.cpu().numpy()
    r = oracle_reference(dspec, inst[0])
    G = steps_per_interval(stats, dspec)
    assert rel(mm[1], mm[0] @ R.T) <= TOL
    assert rel(dd[1], dd[0] @ R.T) <= 2 * dtol(r, 1e-10, G=G)   # two GPU solves, each within the bar


def test_bad_and_empty_inputs(fp):
    dspec, inst = workloads.single_instance_workload()
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-9, stages=3), 10)
    m, dm, st, stats = fp.solve(ctx, inst[:0])           # n == 0: no-op
    bad = np.concatenate([inst, inst, inst])
    bad[0]["L"] = 1
    bad[1]["d"] = -1.0
    bad[2]["L"] = 11                                     # above the context's L_max
    m, dm, st, stats = fp.solve(ctx, bad)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 5).all()
    assert float(m.abs().max()) == 0.0 and float(dm.abs().max()) == 0.0


def test_step_budget_is_reported_not_hung(fp):
    dspec, inst = workloads.single_instance_workload()
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-9, stages=3, max_steps=50), 10)
    m, dm, st, stats = fp.solve(ctx, inst)
    torch.cuda.synchronize()
    assert int(st[0]) == 1                               # FP_STATUS_MAXSTEPS
    assert int(stats[0, 0]) + int(stats[0, 1]) <= 50


def test_phi_hat_matches_oracle_dft(fp):
    """fp_signal (Sec. 2.2 phi_hat, rectangle rule over the last period) equals the
    oracle DFT of the same samples to rounding, and the oracle's own phi_hat
    within the derivative tolerance."""
    from oracle import solve as osolve
    files = sorted(glob.glob(os.path.join(GOLD, "sysmat_L16_v*.npz")))
    ref = np.load(files[0])
    k = int(ref["iy"]) * 32 + int(ref["ix"])
    dspec, inst = workloads.system_matrix_workload()
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-9, stages=3), 16)
    m, dm, st, stats = fp.solve(ctx, inst[k:k + 1])
    G = steps_per_interval(stats, dspec)
    ch = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    out = torch.empty((1, 2, 817, 2), dtype=torch.float64, device=dm.device)
    fp.fp_signal(ctx, dm, 1, 816, ch, out)
    torch.cuda.synchronize()
    ph = out.cpu().numpy()[0]
    ph = ph[..., 0] + 1j * ph[..., 1]
    ph_same = osolve.phi_hat(dm.cpu().numpy()[0], ch, 1632, 816)
    assert np.abs(ph - ph_same).max() <= 1e-12 * np.abs(ph_same).max()
    ph_or = osolve.phi_hat(ref["dmdt"], ch, 1632, 816)
    assert rel(ph, ph_or) <= dtol(ref, 1e-9, "selfconv_phihat", G=G)


def test_tight_tolerance_parity_and_error_against_rtol(fp):
    """The three golden voxels in one 5-stage launch at rtol 1e-9, 1e-10 and
    1e-11: trace, d<m>/dt and phi_hat against the oracle (rtol 1e-12) within
    the derived bars at each tolerance; the errors are printed (-s) for the
    record of error against rtol."""
    from oracle import solve as osolve
    files = sorted(glob.glob(os.path.join(GOLD, "sysmat_L16_v*.npz")))
    refs = [np.load(f) for f in files]
    dspec, inst = workloads.system_matrix_workload()
    ks = [int(r["iy"]) * 32 + int(r["ix"]) for r in refs]
    ch = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    for rtol in (1e-9, 1e-10, 1e-11):
        ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=rtol, stages=5), 16)
        m, dm, st, stats = fp.solve(ctx, inst[ks])
        ph = torch.empty((len(ks), 2, 817, 2), dtype=torch.float64, device=dm.device)
        fp.fp_signal(ctx, dm, len(ks), 816, ch, ph)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        mm, dd, pp = m.cpu().numpy(), dm.cpu().numpy(), ph.cpu().numpy()
        for i, ref in enumerate(refs):
            G = steps_per_interval(stats, dspec, [i])
            e_m, e_d = rel(mm[i], ref["m"]), rel(dd[i], ref["dmdt"])
            e_p = rel(pp[i, ..., 0] + 1j * pp[i, ..., 1], ref["phihat"])
            print("rtol %.0e voxel (%d,%d) G %d: trace %.2e  dm/dt %.2e (bar %.2e)  phi_hat %.2e (bar %.2e)"
                  % (rtol, int(ref["ix"]), int(ref["iy"]), G, e_m, e_d, dtol(ref, rtol, G=G), e_p,
                     dtol(ref, rtol, "selfconv_phihat", G=G)))
            assert e_m <= TOL
            assert e_d <= dtol(ref, rtol, G=G)
            assert e_p <= dtol(ref, rtol, "selfconv_phihat", G=G)
        ctx.close()


@pytest.mark.parametrize("L", [20, 24])
def test_degrees_above_shared_memory_factors(fp, L):
    """Truncation degrees 20 and 24 (blocks of up to 2 L = 48 rows, two row slots
    per lane, FP32 factors in global scratch, 3 stages) against the oracle at
    the same degree (golden, rtol 1e-11, self-convergence against 1e-10): the
    high-degree workload (barrier sigma ~ 11, 12 mT drive, one period), with a
    second instance (sigma ~ 2.8) at degree 14 in the same launch (ragged)."""
    ref = np.load(os.path.join(GOLD, "highdeg_L%d.npz" % L))
    dspec, inst = workloads.high_degree_workload(L)
    low = inst.copy()
    low["K"], low["L"] = 2e3, 14
    both = np.concatenate([inst, low])
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-10, stages=3), 24)
    m, dm, st, stats = fp.solve(ctx, both)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all(), st
    mm, dd = m.cpu().numpy(), dm.cpu().numpy()
    G0, G1 = steps_per_interval(stats, dspec, [0]), steps_per_interval(stats, dspec, [1])
    e_m, e_d = rel(mm[0], ref["m"]), rel(dd[0], ref["dmdt"])
    print("L %d: trace %.2e, dm/dt %.2e (bar %.2e)" % (L, e_m, e_d, dtol(ref, 1e-10, G=G0)))
    assert e_m <= TOL
    assert e_d <= dtol(ref, 1e-10, G=G0)
    r = oracle_reference(dspec, low[0], 1e-12, 1e-11)
    assert rel(mm[1], r["m"]) <= TOL
    assert rel(dd[1], r["dmdt"]) <= dtol(r, 1e-10, G=G1)
    ctx.close()


def test_two_row_slot_path_matches_single_slot_path(fp):
    """The same instances (degrees 10, 14, 16) through the factorisation with
    shared-memory factors and one row slot (context L_max = 16) and through
    the two-row-slot path with global factors (context L_max = 24): both
    integrate the same Galerkin system at the same tolerance, so the traces
    agree within the trace bar and the statuses are OK."""
    dspec = workloads.DriveSpec(amp=(0.010, 0.004, 0.0), freq=(50e3, 50e3, 50e3), phase=(0.0, 0.7, 0.0),
                                period=2e-5, samples_per_period=64, warmup_periods=0, output_periods=1)
    inst = workloads.random_instances(6, 10, seed=21, max_offset=0.006, K_range=(5e2, 3e3))
    inst["L"] = [10, 14, 16, 16, 14, 10]
    out = []
    for Lmax in (16, 24):
        ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-10, stages=3), Lmax)
        m, dm, st, _ = fp.solve(ctx, inst)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all(), (Lmax, st)
        out.append(m.cpu().numpy())
        ctx.close()
    for i in range(len(inst)):
        assert rel(out[1][i], out[0][i]) <= TOL, i

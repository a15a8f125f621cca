"""Discrete adjoint (fp_grad) against central finite differences.

J = sum_{c,k} G_re Re phi_hat + G_im Im phi_hat with seeded random cotangents G;
dJ/d(K, d, theta, phi) from the adjoint kernel versus central differences of
(a) the GPU forward path at a tighter tolerance and (b) the FP64 oracle.  The
adjoint differentiates the recorded step sequence exactly; central differences
(relative step 1e-4) carry O(h^2) truncation and rtol/h noise, so the stated
agreement is 1e-5 relative to the gradient norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2106_08040_gb300 import build, workloads      # noqa: E402

pytestmark = pytest.mark.gpu

DSPEC = workloads.DriveSpec(amp=(0.010, 0.0, 0.0), freq=(50e3, 50e3, 50e3), phase=(0.0, 0.0, 0.0),
                            period=2e-5, samples_per_period=64, warmup_periods=0, output_periods=1)
CH = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
KMAX = 20
L = 8


@pytest.fixture(scope="module")
def fp():
    build.build()
    from paper_2106_08040_gb300 import fp as fpmod
    return fpmod


def instances():
    inst = workloads.random_instances(3, L, seed=5, max_offset=0.004, K_range=(5e2, 3e3))
    return inst


def cotangent(n):
    rng = np.random.default_rng(9)
    return rng.normal(size=(n, 2, KMAX + 1, 2))


def gpu_J(fp, inst, G, rtol):
    ctx = fp.Context(fp.Material(), fp.Drive(**DSPEC.__dict__), fp.Tol(rtol=rtol, stages=3), L)
    m, dm, st, _ = fp.solve(ctx, inst)
    out = torch.empty((len(inst), 2, KMAX + 1, 2), dtype=torch.float64, device=dm.device)
    fp.fp_signal(ctx, dm, len(inst), KMAX, CH, out)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    return (out.cpu().numpy() * G).sum(axis=(1, 2, 3))


def perturbed(inst, p, h):
    a, b = inst.copy(), inst.copy()
    key = ["K", "d", "theta", "phi"][p]
    step = h * abs(inst[key]) if p < 2 else np.full(len(inst), h)
    a[key] = inst[key] + step
    b[key] = inst[key] - step
    return a, b, step


def adjoint(fp, inst, G, rtol=1e-10):
    ctx = fp.Context(fp.Material(), fp.Drive(**DSPEC.__dict__), fp.Tol(rtol=rtol, stages=3), L)
    n = len(inst)
    dev = torch.device("cuda")
    d_inst = fp.instances_to_device(inst, dev)
    dJ = torch.from_numpy(np.ascontiguousarray(G)).to(dev)
    grad = torch.empty((n, 4), dtype=torch.float64, device=dev)
    st = torch.empty((n,), dtype=torch.int32, device=dev)
    stats = torch.empty((n, 4), dtype=torch.int32, device=dev)
    work = torch.empty(fp.fp_grad_workspace_bytes(ctx, n), dtype=torch.uint8, device=dev)
    fp.fp_grad(ctx, d_inst, n, KMAX, CH, dJ, grad, st, work, d_stats=stats)
    torch.cuda.synchronize()
    return grad.cpu().numpy(), st.cpu().numpy(), stats.cpu().numpy()


def test_adjoint_vs_gpu_central_differences(fp):
    inst = instances()
    G = cotangent(len(inst))
    g, st, stats = adjoint(fp, inst, G)
    assert (st == 0).all(), (st, stats)
    assert (stats[:, 0] > 64).all()            # several checkpoint segments
    fd = np.zeros_like(g)
    for p in range(4):
        a, b, step = perturbed(inst, p, 1e-4)
        fd[:, p] = (gpu_J(fp, a, G, 1e-11) - gpu_J(fp, b, G, 1e-11)) / (2 * step)
    for i in range(len(inst)):
        scale = np.linalg.norm(fd[i] * np.array([inst[i]["K"], inst[i]["d"], 1.0, 1.0]))
        err = np.abs((g[i] - fd[i]) * np.array([inst[i]["K"], inst[i]["d"], 1.0, 1.0]))
        assert err.max() <= 1e-5 * scale, (i, g[i], fd[i])


def test_adjoint_vs_oracle_central_differences(fp):
    from oracle import physics, solve
    inst = instances()[:1]
    G = cotangent(1)
    g, st, _ = adjoint(fp, inst, G)
    assert st[0] == 0
    drive = physics.Drive(amp=DSPEC.amp, freq=DSPEC.freq, phase=DSPEC.phase, period=DSPEC.period)
    sched = solve.Schedule(64, 0, 1)

    def J(rec):
        oi = solve.Instance(h_off=tuple(rec["h_off"]), theta=float(rec["theta"]), phi=float(rec["phi"]),
                            K=float(rec["K"]), d=float(rec["d"]), L=L)
        r = solve.solve_instance(physics.Material(), drive, oi, sched, rtol=1e-12)
        ph = solve.phi_hat(r["dmdt"], CH, 64, KMAX)
        return float((ph.real * G[0, :, :, 0]).sum() + (ph.imag * G[0, :, :, 1]).sum())

    fd = np.zeros(4)
    for p in range(4):
        a, b, step = perturbed(inst, p, 1e-4)
        fd[p] = (J(a[0]) - J(b[0])) / (2 * step[0])
    w = np.array([inst[0]["K"], inst[0]["d"], 1.0, 1.0])
    assert np.abs((g[0] - fd) * w).max() <= 1e-5 * np.linalg.norm(fd * w), (g[0], fd)


def test_autograd_function_matches_fp_grad(fp):
    inst = instances()
    G = cotangent(len(inst))
    g_ref, st, _ = adjoint(fp, inst, G)
    ctx = fp.Context(fp.Material(), fp.Drive(**DSPEC.__dict__), fp.Tol(rtol=1e-10, stages=3), L)
    dev = torch.device("cuda")
    params = torch.tensor(np.stack([inst["K"], inst["d"], inst["theta"], inst["phi"]], 1), dtype=torch.float64,
                          device=dev, requires_grad=True)
    h_off = torch.tensor(inst["h_off"], dtype=torch.float64, device=dev)
    ph = fp.phi_hat(params, h_off, ctx, L, KMAX, CH)
    loss = (ph * torch.from_numpy(G).to(dev)).sum()
    loss.backward()
    np.testing.assert_allclose(params.grad.cpu().numpy(), g_ref, rtol=1e-9, atol=0)


@pytest.mark.parametrize("stages", [3, 5])
def test_adjoint_L16_lissajous_vs_gpu_central_differences(fp, stages):
    """Where the gradients are used: system-matrix voxels 0 and 1 (L = 16,
    cosine Lissajous drive, 1 warm-up + 1 output period, 1632 samples, all 817
    harmonics of both channels in J).  Both have transposed stage solves that
    stagnate near the single-precision level of the factor solves.  The
    adjoint (3 or 5 stages, rtol 1e-10; with 5 stages its factors live in the
    workspace) against central differences (relative step 1e-4) of the 5-stage
    forward at rtol 1e-11: within 1e-5 of the gradient norm per parameter."""
    dspec, inst = workloads.system_matrix_workload()
    inst = inst[:2]
    n, K = len(inst), 816
    ch = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    G = np.random.default_rng(3).normal(size=(n, 2, K + 1, 2))
    dev = torch.device("cuda")
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__),
                     fp.Tol(rtol=1e-10, stages=stages, max_steps=400000), 16)
    grad = torch.empty((n, 4), dtype=torch.float64, device=dev)
    st = torch.empty((n,), dtype=torch.int32, device=dev)
    stats = torch.empty((n, 4), dtype=torch.int32, device=dev)
    work = torch.empty(fp.fp_grad_workspace_bytes(ctx, n), dtype=torch.uint8, device=dev)
    fp.fp_grad(ctx, fp.instances_to_device(inst, dev), n, K, ch, torch.from_numpy(G).to(dev), grad, st, work,
               d_stats=stats)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all(), (st, stats)
    g = grad.cpu().numpy()
    ctx5 = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-11, stages=5), 16)
    recs, steps = [], []
    for i in range(n):
        for p in range(4):
            a, b, step = perturbed(inst[i:i + 1], p, 1e-4)
            recs += [a, b]
            steps.append(step[0])
    allr = np.concatenate(recs)
    _, dm, st5, _ = fp.solve(ctx5, allr, want_m=False)
    ph = torch.empty((len(allr), 2, K + 1, 2), dtype=torch.float64, device=dev)
    fp.fp_signal(ctx5, dm, len(allr), K, ch, ph)
    torch.cuda.synchronize()
    assert (st5.cpu().numpy() == 0).all()
    ph = ph.cpu().numpy()
    for i in range(n):
        fd = np.array([((ph[8 * i + 2 * p] - ph[8 * i + 2 * p + 1]) * G[i]).sum() / (2 * steps[4 * i + p])
                       for p in range(4)])
        w = np.array([inst[i]["K"], inst[i]["d"], 1.0, 1.0])
        assert np.abs((g[i] - fd) * w).max() <= 1e-5 * np.linalg.norm(fd * w), (i, g[i], fd)

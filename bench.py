#!/usr/bin/env python
"""Throughput of the batched Neel Fokker-Planck solve on GB300.

Workload (default): the 32 x 32-voxel system-matrix batch -- cosine Lissajous
drive 12 mT per axis, f_x = 2.5 MHz/102, f_y = 2.5 MHz/96, 1632 samples per
652.8 us period, selection gradient diag(-1, -1, 2) T/m over 24 x 24 mm, easy
axis along x, K = 2e3 J/m^3, d = 20 nm, truncation L = 16; every instance is
integrated over 1 warm-up + 1 output period (2 instance-periods) and its
phi_hat harmonics computed.  One step = fp_solve_batch + fp_signal over the
batch, inputs resident in HBM.  Metric: instance-periods/s (whole job).

Multi-GPU (torchrun, one rank per GPU): weak scaling, rank r solves the same
voxel batch for easy-axis angle vartheta_r = 15 deg * r (the paper's angle set),
no collective on the data path; barrier + max-over-ranks timing.

--impl reference times the FP64 CPU oracle (the reference arm) on
a bounded sample of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FP instance-periods/s at ≤1e-9 rel err vs FP64 oracle; surrogate speedup at 1e-3"
UNIT = "instance-periods/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--stages", type=int, default=5, help="Radau IIA stages: 5 (order 9) or 3 (order 5)")
    p.add_argument("--rtol", type=float, default=1e-9)
    p.add_argument("--cpu-sample-s", type=float, default=20.0, help="target CPU seconds per oracle process")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--instances", type=int, default=0, help="profiling: first N voxels only (0 = all)")
    p.add_argument("--warmup-periods", type=int, default=1, help="profiling: warm-up periods per instance")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-surrogate", action="store_true", help="skip the surrogate measurement")
    p.add_argument("--no-sweep", action="store_true", help="skip the uneven-sweep measurement")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    p.add_argument("--adjoint-stages", type=int, default=3, choices=(3, 5), help="Radau stages of the adjoint leg")
    p.add_argument("--no-models", action="store_true", help="skip the M0/M1/M2 model measurement")
    p.add_argument("--m1-dictionary", type=int, default=96, help="M1 fit: dictionary elements per call")
    p.add_argument("--m2-tuples", type=int, default=96, help="M2: (D, K) tuples in the dictionary")
    p.add_argument("--sweep-instances", type=int, default=2048)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_for_rank(rank, args):
    from paper_2106_08040_gb300 import workloads
    dspec, inst = workloads.system_matrix_workload()
    inst["phi"] = np.deg2rad(15.0 * (rank % 12))
    if args.instances:
        inst = inst[:args.instances]
    if args.warmup_periods != dspec.warmup_periods:
        d = dict(dspec.__dict__)
        d["warmup_periods"] = args.warmup_periods
        dspec = workloads.DriveSpec(**d)
    return dspec, inst


def max_over_ranks(x, dist, device):
    """Max of a per-rank scalar over the process group (the slowest rank's time)."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_per_rank, periods, ms):
    """Whole-job instance-periods/s: every rank solves its own n instances."""
    return world * n_per_rank * periods / (ms * 1e-3)


# ----------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only queries)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------- flop accounting ----
def fp64_flops_per_instance(stats, N, nnz, S):
    """Algorithmic FP64 flops of one instance from the kernel's own counters:
    every Newton iteration applies A at S stage values (2 nnz each) and forms
    S residuals (S^2 + S multiply-adds per entry) and S stage updates; every
    accepted or rejected step adds the error combination (S + 1 per entry),
    and every accepted step one more apply for f(t, y) and the state update."""
    steps, rej, iters = stats[:, 0].astype(np.float64), stats[:, 1].astype(np.float64), stats[:, 2].astype(np.float64)
    per_iter = S * 2.0 * nnz + N * (2.0 * S * S + 3.0 * S)
    per_try = N * 2.0 * (S + 1)
    per_acc = 2.0 * nnz + N
    return iters * per_iter + (steps + rej) * per_try + steps * per_acc


def operator_nnz(fp, L):
    A = fp.fp_operator_dense(fp.Material(), L, 2e3, 20e-9, [0.003, -0.002, 0.004])
    return int(np.count_nonzero(A))


# -------------------------------------------------------------- CPU oracle ----
def _oracle_window(args):
    """One bounded oracle solve: voxel rec of the workload, ns samples starting at
    output sample j0.  Setup (weak-form matrices) and the start state (Boltzmann
    density at the window's start field) are not timed."""
    import os as _os
    _os.environ.setdefault("OMP_NUM_THREADS", "1")
    (dspec_d, rec, j0, ns, rtol) = args
    from oracle import galerkin, physics, radau, solve
    drive = physics.Drive(amp=dspec_d["amp"], freq=dspec_d["freq"], phase=dspec_d["phase"], period=dspec_d["period"])
    inst = solve.Instance(h_off=tuple(rec["h_off"]), theta=float(rec["theta"]), phi=float(rec["phi"]),
                          K=float(rec["K"]), d=float(rec["d"]), L=int(rec["L"]))
    P = physics.derive(physics.Material(), inst.K, inst.d)
    n = physics.easy_axis(inst.theta, inst.phi)
    A0, A1 = galerkin.weak_form_matrices(inst.L, P, n)
    off = np.asarray(inst.h_off)

    def A_of_t(t):
        B = drive.field(t, off)
        return A0 + B[0] * A1[0] + B[1] * A1[1] + B[2] * A1[2]

    S = dspec_d["samples_per_period"]
    T_s = drive.period / S
    t_start = (dspec_d["warmup_periods"] + j0 / S) * drive.period
    c_start = galerkin.boltzmann_coeffs(inst.L, P, n, drive.field(t_start, off))
    t_out = t_start + (np.arange(ns) + 1) * T_s
    integ = radau.RadauIIA(A_of_t, rtol=rtol, h0=min(T_s, 0.01 * P.tau), h_max=T_s)
    t0 = time.time()
    integ.integrate(t_start, c_start, t_out)
    return time.time() - t0, ns / S, integ.n_steps


def cpu_oracle_sample(dspec, inst, target_s, rtol=1e-12):
    """Oracle (its defining tolerance, rtol 1e-12) on all host cores, one
    single-threaded process per core, each timing a window of output samples of
    one voxel; the windows start at evenly spread positions of the output period,
    so together they cover its field sweep.  Throughput is extrapolated linearly
    by sample count to instance-periods/s (one instance-period = S samples)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    S = dspec.samples_per_period
    dd = dict(amp=dspec.amp, freq=dspec.freq, phase=dspec.phase, period=dspec.period, samples_per_period=S,
              warmup_periods=dspec.warmup_periods)
    rng = np.random.default_rng(0)
    picks = rng.choice(len(inst), size=cores, replace=cores > len(inst))
    starts = [(q * S) // cores for q in range(cores)]
    el, _, _ = _oracle_window((dd, inst[picks[0]], starts[0], 2, rtol))      # calibration: 2 samples
    per_sample = max(el / 2, 1e-3)
    ns = int(max(2, min(S // cores, target_s / per_sample)))
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"                         # children: single-threaded BLAS, one per core
    try:
        with ctx.Pool(cores) as pool:
            res = pool.map(_oracle_window, [(dd, inst[k], j0, ns, rtol) for k, j0 in zip(picks, starts)])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    # each process solves its own window: the job rate is the sum of the per-process rates
    rate = sum(r[1] / r[0] for r in res)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "extrapolated": True,
            "sample": "%d voxels of the 32x32 L=16 batch, one window of %d output samples each, windows at %d evenly "
                      "spread positions of the output period (Radau IIA rtol 1e-12, one process per core; setup and "
                      "the window's start state untimed); %d oracle steps in %.1f s of CPU; instance-periods/s "
                      "extrapolated by sample count" % (cores, ns, cores, sum(r[2] for r in res), sum(r[0] for r in res))}


# --------------------------------------------------------------- surrogate --
SUR_FLOPS_PER_QUERY = 2.0 * (7 * 512 + 3 * 512 * 512 + 512 * 800)   # algorithmic (unpadded input)


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured (MEASURED_PEAKS.json %s)" % key
    except Exception:
        return fallback, "fallback"


def surrogate_leg(fp, dev):
    """Trained surrogate ensemble: inference throughput on the 40^3 x 16
    (1,024,000-query) grid, and its error and speed against the FP solve on
    fresh draws from its training domain."""
    import torch
    from paper_2106_08040_gb300 import surrogate, surrogate_train as stt, workloads
    path = stt.DEFAULT_OUT
    base, ext = os.path.splitext(path)
    if not os.path.exists("%s.m0%s" % (base, ext)):
        return {"unavailable": "no trained weights at %s" % os.path.relpath(path, ROOT)}
    ens = stt.Ensemble.load(path, device=dev)
    # query grid: 40^3 offsets over a 24 mm cube (gradient diag(-1, -1, 2) T/m) x 16 Fibonacci axes
    g = -12e-3 + (np.arange(40) + 0.5) * 24e-3 / 40
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    off = np.stack([-X.ravel(), -Y.ravel(), 2 * Z.ravel()], 1)
    th, ph = workloads.fibonacci_directions(16)
    q = off.shape[0] * 16
    rng = np.random.default_rng(5)
    xq = np.empty((q, 7), dtype=np.float32)
    xq[:, 0:3] = np.repeat(off, 16, axis=0)
    xq[:, 3] = np.tile(th, off.shape[0])
    xq[:, 4] = np.tile(ph, off.shape[0])
    xq[:, 5] = rng.uniform(np.log(5e2), np.log(1e4), size=q)            # ln K, K log-uniform
    xq[:, 6] = np.log(20e-9) + 0.1 * rng.normal(size=q)                 # ln d, d log-normal
    x = torch.from_numpy(xq).to(dev)
    for _ in range(3):
        ens.infer(x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        ens.infer(x)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    q_per_s = q / (ms * 1e-3)
    # error reference: fresh draws from the training domain, solved by the FP path
    draw = workloads.uneven_sweep_instances(1024, 16, seed=7)
    draw = draw[fp.Material().sigma(draw["K"], draw["d"]) <= 12.0][:152]
    ctx = stt.solver_context(16, 1e-7)
    torch.cuda.synchronize()
    t0 = time.time()
    y, st = stt.solve_signals(ctx, draw)
    t_solve = time.time() - t0
    ctx.close()
    ok = st == 0
    mean, spread = ens.infer(torch.from_numpy(surrogate.features(draw).astype(np.float32)).to(dev))
    err = stt.relative_errors(mean.cpu().numpy().astype(np.float64)[ok], y[ok])
    spr = spread.cpu().numpy()[ok]
    solver_per_s = len(draw) / t_solve
    peak, src = measured_peak("bf16_tflops", 1900.0)
    achieved = 2 * SUR_FLOPS_PER_QUERY * q / (ms * 1e-3) / 1e12
    gate = {}
    for g_thr in (1e-3, 1e-2, 3e-2, 1e-1):
        acc = spr <= g_thr
        f_rej = 1.0 - acc.mean()
        t_per_q = 1.0 / q_per_s + f_rej / solver_per_s
        gate["%g" % g_thr] = {"accepted": float(acc.mean()),
                              "err_p90_accepted": float(np.quantile(err[acc], 0.9)) if acc.any() else None,
                              "speedup_with_fallback": float((1.0 / solver_per_s) / t_per_q)}
    return {"queries": q, "ms": ms, "queries_per_s": q_per_s, "ensemble": 2,
            "solver_instances_per_s": solver_per_s, "speedup_vs_solver": q_per_s / solver_per_s,
            "holdout": int(ok.sum()), "rel_err_median": float(np.median(err)),
            "rel_err_p90": float(np.quantile(err, 0.9)), "gate_on_member_spread": gate,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_source": src,
                         "kernel": "mlp_gemm_kernel (tcgen05 BF16, 2 members x 5 layers)"},
            "error_reference": "fp_solve_batch + fp_signal, L = 16, rtol 1e-7, 152 fresh draws of the training domain"}


def adjoint_leg(fp, dev, n_inst=152, stages=3):
    """Discrete adjoint (fp_grad) on the first voxels of the system-matrix batch:
    gradients dJ/d(K, d, theta, phi) of a seeded linear functional of phi_hat,
    timed against the forward solve + phi_hat of the same instances."""
    import torch
    from paper_2106_08040_gb300 import workloads
    dspec, inst = workloads.system_matrix_workload()
    inst = inst[:n_inst]
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-9, stages=stages, max_steps=200000), 16)
    n, K = len(inst), 816
    ch = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    d_inst = fp.instances_to_device(inst, dev)
    dJ = torch.from_numpy(np.random.default_rng(3).normal(size=(n, 2, K + 1, 2))).to(dev)
    grad = torch.empty((n, 4), dtype=torch.float64, device=dev)
    st = torch.empty((n,), dtype=torch.int32, device=dev)
    gstats = torch.zeros((n, 4), dtype=torch.int32, device=dev)
    work = torch.empty(fp.fp_grad_workspace_bytes(ctx, n), dtype=torch.uint8, device=dev)
    S = ctx.num_samples()
    dm = torch.empty((n, S, 3), dtype=torch.float64, device=dev)
    ph = torch.empty((n, 2, K + 1, 2), dtype=torch.float64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    fp.fp_solve_batch(ctx, d_inst, n, None, dm, st, None)
    fp.fp_signal(ctx, dm, n, K, ch, ph)
    ev[1].record()
    fp.fp_grad(ctx, d_inst, n, K, ch, dJ, grad, st, work, d_stats=gstats)
    ev[2].record()
    torch.cuda.synchronize()
    t_f, t_a = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    periods = dspec.warmup_periods + dspec.output_periods
    # gradient error: central differences (relative step 1e-4) of the 5-stage
    # forward at rtol 1e-11 on the first two voxels
    g = grad.cpu().numpy()
    Gh = dJ.cpu().numpy()
    ctx5 = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=1e-11, stages=5), 16)
    recs, steps = [], []
    for i in (0, 1):
        for p, key in enumerate(["K", "d", "theta", "phi"]):
            for sgn in (1, -1):
                r = inst[i:i + 1].copy()
                h = 1e-4 * abs(float(r[key][0])) if p < 2 else 1e-4
                r[key] = r[key] + sgn * h
                recs.append(r)
                steps.append(h)
    allr = np.concatenate(recs)
    _, dmf, stf, _ = fp.solve(ctx5, allr, want_m=False)
    phf = torch.empty((len(allr), 2, K + 1, 2), dtype=torch.float64, device=dev)
    fp.fp_signal(ctx5, dmf, len(allr), K, ch, phf)
    torch.cuda.synchronize()
    phf = phf.cpu().numpy()
    rel_err = []
    for a, i in enumerate((0, 1)):
        fd = np.array([((phf[a * 8 + 2 * p] - phf[a * 8 + 2 * p + 1]) * Gh[i]).sum() / (2 * steps[a * 8 + 2 * p])
                       for p in range(4)])
        w = np.array([inst[i]["K"], inst[i]["d"], 1.0, 1.0])
        rel_err.append((np.abs((g[i] - fd) * w) / np.linalg.norm(fd * w)).tolist())
    ctx5.close()
    out = {"instances": n, "radau_stages": stages, "forward_ms": t_f, "adjoint_ms": t_a, "adjoint_over_forward": t_a / t_f,
           "gradients_per_s": n / (t_a * 1e-3), "instance_periods_per_s": n * periods / (t_a * 1e-3),
           "adjoint_fit_iteration_s_extrapolated": 64 * 1024 / (n / (t_a * 1e-3)),
           "adjoint_fit_iteration_note": "64 candidate sets x 32 x 32 voxels = 65,536 gradient evaluations of this "
                                         "workload per iteration, at the measured gradient rate (persistent CTAs: "
                                         "the workspace does not grow with n)",
           "status_ok": int((st.cpu().numpy() == 0).sum()), "workspace_bytes": int(work.numel()),
           "failed_phase_counts": np.bincount(gstats[:, 2].cpu().numpy(), minlength=4).tolist(),
           "grad_rel_err_vs_central_differences": {"voxels": [0, 1], "per_parameter": rel_err,
                                                   "max": float(np.max(rel_err)),
                                                   "reference": "central differences, relative step 1e-4, of "
                                                                "fp_solve_batch + fp_signal at rtol 1e-11 (5 stages); "
                                                                "error in units of the gradient norm"},
           "workload": "first %d voxels of the 32x32 system-matrix batch, L = 16, Radau s = %d, rtol 1e-9, "
                       "checkpoints every 64 steps" % (n, stages)}
    ctx.close()
    return out


def models_leg(fp, dev, peak64, Q=96, J2=96):
    """Sec. 2.2 models on the system-matrix grid: M0 traces + phi_hat for the
    1024 voxels, and the M1 fit of a Q-element dictionary (8 diameters x 12
    anisotropies at one angle, synthetic phi_hat of the solver's shape) against
    one measured matrix.  fp_m1_fit reads the dictionary twice (filter, then
    row errors): HBM-bound."""
    import torch
    from paper_2106_08040_gb300 import workloads
    dspec, inst = workloads.system_matrix_workload()
    ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(), 8)
    n, S, K1, C = len(inst), ctx.num_samples(), 817, 2
    d_inst = fp.instances_to_device(inst, dev)
    dm = torch.empty((n, S, 3), dtype=torch.float64, device=dev)
    ph = torch.empty((n, C, K1, 2), dtype=torch.float64, device=dev)
    ch = [[1.0, 0, 0], [0, 1.0, 0]]
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(2):
        fp.fp_equilibrium(ctx, d_inst, n, None, dm)
        fp.fp_signal(ctx, dm, n, K1 - 1, ch, ph)
    e[0].record()
    fp.fp_equilibrium(ctx, d_inst, n, None, dm)
    fp.fp_signal(ctx, dm, n, K1 - 1, ch, ph)
    e[1].record()
    gen = torch.Generator(device=dev)
    gen.manual_seed(1)
    phi = torch.randn((Q, n, C, K1, 2), dtype=torch.float64, device=dev, generator=gen)
    Sm = torch.randn((n, C, K1, 2), dtype=torch.float64, device=dev, generator=gen)
    a = torch.empty((Q, C, K1, 2), dtype=torch.float64, device=dev)
    eps = torch.empty((Q, C, K1), dtype=torch.float64, device=dev)
    smax = torch.empty((C, K1), dtype=torch.float64, device=dev)
    for _ in range(2):
        fp.fp_m1_fit(phi, Q, Sm, n, C, K1, a, eps, smax)
    torch.cuda.synchronize()
    reps = 5
    e[2].record()
    for _ in range(reps):
        fp.fp_m1_fit(phi, Q, Sm, n, C, K1, a, eps, smax)
    e[3].record()
    torch.cuda.synchronize()
    ms_m0 = e[0].elapsed_time(e[1])
    ms_m1 = e[2].elapsed_time(e[3]) / reps
    by = 2.0 * (phi.numel() + Sm.numel()) * 8 + (a.numel() + eps.numel()) * 8
    hbm, src = measured_peak("hbm_gbs", 6800.0)
    # FP64 work per (element, dictionary entry): S conj(Phi) (8), |Phi|^2 (4) and
    # |S|^2 (3) in the first pass; a Phi (6), S - a Phi (2), |r|^2 (4) in the second
    fl = 27.0 * Q * n * C * K1
    out = {"m0_voxels": n, "m0_ms": ms_m0, "m0_voxel_periods_per_s": n * 2 / (ms_m0 * 1e-3),
           "m1_dictionary": Q, "m1_ms": ms_m1, "m1_fits_per_s": Q / (ms_m1 * 1e-3),
           "m1_roofline": {"bound": "alu", "achieved": fl / (ms_m1 * 1e-3) / 1e12, "peak": peak64, "unit": "TFLOP/s",
                           "frac": fl / (ms_m1 * 1e-3) / 1e12 / peak64,
                           "peak_source": "measured FP64 FMA throughput (fp_peak_fp64, this run)",
                           "hbm_GBps": by / (ms_m1 * 1e-3) / 1e9, "hbm_frac": by / (ms_m1 * 1e-3) / 1e9 / hbm,
                           "hbm_peak_source": src, "bytes_per_launch": by,
                           "kernel": "fp_m1_pass1 + fp_m1_pass2 (FP64-pipe bound on GB300)"}}
    ctx.close()
    del phi, Sm
    # M2 at the paper's shapes: 12 angles, an 11 x 11 voxel grid, J = 8 x 12
    # (D, K) tuples, both channels, rows I_freq (mixing orders up to 20)
    A2, N2 = 12, 121
    ks = fp.fp_freq_index_set(20, 20, 16, K1 - 1)
    phi2 = torch.randn((A2, J2, N2, C, K1, 2), dtype=torch.float64, device=dev, generator=gen)
    a2 = torch.randn((A2, J2, C, K1, 2), dtype=torch.float64, device=dev, generator=gen)
    S2 = torch.randn((A2, N2, C, K1, 2), dtype=torch.float64, device=dev, generator=gen)
    smax2 = torch.sqrt((S2 ** 2).sum(-1)).amax(1).contiguous()
    d_ks = torch.from_numpy(ks.astype(np.int32)).to(dev)
    G = torch.empty((J2 + 1, J2 + 1, 2), dtype=torch.float64, device=dev)
    fp.fp_m2_gram(phi2, a2, S2, smax2, A2, J2, N2, C, K1, d_ks, len(ks), G)
    torch.cuda.synchronize()
    e[0].record()
    fp.fp_m2_gram(phi2, a2, S2, smax2, A2, J2, N2, C, K1, d_ks, len(ks), G)
    e[1].record()
    torch.cuda.synchronize()
    ms_g = e[0].elapsed_time(e[1])
    t0 = time.time()
    w, obj, res, sv, srank = fp.fp_m2_solve(G.cpu().numpy(), J2, 21)
    t_host = time.time() - t0
    rows = A2 * N2 * C * len(ks)
    tiles = -(-(J2 + 1) // 16)
    flops = 8.0 * rows * (16 * 16) * tiles * (tiles + 1) / 2      # complex multiply-adds of the computed tiles
    flops_alg = 8.0 * rows * (J2 + 1) * (J2 + 2) / 2              # upper triangle of the Gram matrix
    out.update({"m2_gram_ms": ms_g, "m2_rows": rows, "m2_J": J2, "m2_angles": A2, "m2_voxels": N2,
                "m2_host_solve_s": t_host, "m2_rank": srank, "m2_nonzero_weights": int((w > 1e-12 * w.max()).sum()),
                "m2_gram_roofline": {"bound": "alu", "achieved": flops_alg / (ms_g * 1e-3) / 1e12, "peak": peak64,
                                     "unit": "TFLOP/s", "frac": flops_alg / (ms_g * 1e-3) / 1e12 / peak64,
                                     "executed_over_algorithmic": flops / flops_alg,
                                     "kernel": "fp_m2_gram_kernel (FP64, upper-triangle tiles)"}})
    del phi2, a2, S2
    return out


STATUS_NAMES = {1: "MAXSTEPS", 2: "STEP_UNDERFLOW", 3: "NONFINITE", 4: "NEWTON_FAIL", 5: "BAD_INPUT", 6: "UNRESOLVED"}


def sweep_leg(fp, dev, n_inst):
    """Uneven sweep: draws of the uneven-sweep distribution (64 x 64 voxel
    offsets, 16 Fibonacci axes, K log-uniform, d log-normal) with L per
    instance from the truncation rule (8..16), planned, autotuned and run as
    one graph; instance-periods/s."""
    import torch
    from paper_2106_08040_gb300 import workloads
    dspec = workloads.drive_lissajous()
    drv = fp.Drive(**dspec.__dict__)
    draw = workloads.uneven_sweep_instances(n_inst, 24, seed=11)
    draw["L"] = fp.truncation_degree(draw, drive=drv, L_min=8, L_max=24)
    ctx = fp.Context(fp.Material(), drv, fp.Tol(rtol=1e-9, stages=3), 24)
    n = len(draw)
    S = ctx.num_samples()
    d_inst = fp.instances_to_device(draw, dev)
    m = torch.empty((n, S, 3), dtype=torch.float64, device=dev)
    dm = torch.empty_like(m)
    st = torch.empty((n,), dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(device=dev)
    sw = fp.Sweep(ctx, draw, bucket_width=2)
    t0 = time.time()
    with torch.cuda.stream(s):
        sw.autotune(d_inst, m, dm, st, sample=32, stream=s)
    s.synchronize()
    t_tune = time.time() - t0
    with torch.cuda.stream(s):
        sw.run(d_inst, m, dm, st, stream=s)            # capture
    s.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        e0.record(s)
        sw.run(d_inst, m, dm, st, stream=s)            # graph replay
        e1.record(s)
    s.synchronize()
    ms = e0.elapsed_time(e1)
    status = st.cpu().numpy()
    periods = dspec.warmup_periods + dspec.output_periods
    per_L = {}
    for Lv in np.unique(draw["L"]):
        sel = draw["L"] == Lv
        codes = np.bincount(status[sel], minlength=7)
        per_L[int(Lv)] = {"instances": int(sel.sum()), "ok": int((status[sel] == 0).sum()),
                          "unresolved": int((status[sel] == 6).sum()),
                          "other": int(((status[sel] != 0) & (status[sel] != 6)).sum()),
                          "other_by_status": {STATUS_NAMES.get(c, str(c)): int(codes[c])
                                              for c in range(len(codes)) if c not in (0, 6) and codes[c]}}
    out = {"instances": n, "per_degree": per_L,
           "ms": ms, "instance_periods_per_s": n * periods / (ms * 1e-3), "status_ok": int((status == 0).sum()),
           "status_unresolved": int((status == 6).sum()), "autotune_s": t_tune, "buckets": sw.info(),
           "workload": "uneven-sweep distribution (64 x 64 offsets, 16 Fibonacci axes, K log-uniform 5e2-1e4, "
                       "d log-normal 20 nm), no barrier cap, L by the truncation rule in [8, 24], Lissajous drive, "
                       "1 warm-up + 1 output period, rtol 1e-9, 3 stages above degree 16"}
    sw.close()
    ctx.close()
    return out


# ------------------------------------------------------------------ GPU arm --
def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2106_08040_gb300 import build
    rank, world, local = dist_env()
    if world > 1:
        os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    from paper_2106_08040_gb300 import fp
    dspec, inst = workload_for_rank(rank, args)
    n = len(inst)
    L = int(inst["L"][0])
    drv = fp.Drive(**dspec.__dict__)
    tol = fp.Tol(rtol=args.rtol, stages=args.stages)
    ctx = fp.Context(fp.Material(), drv, tol, L)
    S_out = ctx.num_samples()
    K = 816
    C = 2
    ch = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    dev = torch.device("cuda", local)
    d_inst = fp.instances_to_device(inst, dev)
    m = torch.empty((n, S_out, 3), dtype=torch.float64, device=dev)
    dm = torch.empty_like(m)
    st = torch.empty((n,), dtype=torch.int32, device=dev)
    stats = torch.empty((n, 4), dtype=torch.int32, device=dev)
    ph = torch.empty((n, C, K + 1, 2), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        fp.fp_solve_batch(ctx, d_inst, n, m, dm, st, stats, stream=stream)
        fp.fp_signal(ctx, dm, n, K, ch, ph, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    peak = fp.fp_peak_fp64()
    nnz = operator_nnz(fp, L)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))                        # evict L2 between timed steps (not timed)
        a, b, c = ev[k]
        a.record(stream)
        fp.fp_solve_batch(ctx, d_inst, n, m, dm, st, stats, stream=stream)
        b.record(stream)
        fp.fp_signal(ctx, dm, n, K, ch, ph, stream=stream)
        c.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    solve_ms = [a.elapsed_time(b) for a, b, c in ev]
    ms = sum(step_ms) / args.steps
    t_solve = sum(solve_ms) / args.steps
    if world > 1:
        ms = max_over_ranks(ms, dist, dev)
    status = st.cpu().numpy()
    sts = stats.cpu().numpy()
    periods = drv.warmup_periods + drv.output_periods
    value = job_throughput(world, n, periods, ms)
    # roofline of the dominant kernel (the solver): FP64 pipe
    flops = float(fp64_flops_per_instance(sts, (L + 1) ** 2, nnz, args.stages).sum())
    achieved = flops / (t_solve * 1e-3) / 1e12
    # DRAM traffic is not measured inside the run (it needs a profiler): null
    roof = {"bound": "alu", "achieved": achieved, "peak": peak / 1e3, "unit": "TFLOP/s",
            "frac": achieved / (peak / 1e3), "traffic": None,
            "kernel": "fp_solve_kernel<%d> (FP64 pipe)" % args.stages,
            "peak_source": "measured FP64 FMA throughput (fp_peak_fp64, this GPU, this run)"}
    # end-to-end through the public API: host instances -> solve -> phi_hat -> host
    h_inst = torch.from_numpy(np.ascontiguousarray(inst).view(np.uint8).reshape(-1).copy()).pin_memory()
    h_ph = torch.empty(ph.shape, dtype=ph.dtype).pin_memory()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_ms = float("nan")
    if not args.no_e2e:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            d_inst.copy_(h_inst, non_blocking=True)
            step()
            h_ph.copy_(ph, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "system_matrix_32x32_L16_lissajous" if n == 1024 and periods == 2 else
                       "system_matrix_L16_lissajous_subset(%d instances, %d periods)" % (n, periods),
                       "instances_per_gpu": n, "L": L,
                       "periods_per_instance": periods, "samples_per_period": drv.samples_per_period,
                       "radau_stages": args.stages, "rtol": args.rtol, "harmonics": K + 1, "channels": C,
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "parallelism": "independent instances; weak scaling, rank r uses easy-axis angle 15 deg*r"},
            "gpu_launches": 2 * args.steps,
            "e2e": {"value": job_throughput(world, n, periods, e2e_ms) if e2e_ms == e2e_ms else None, "unit": UNIT,
                    "h2d_bytes_per_step": int(h_inst.numel()), "d2h_bytes_per_step": int(h_ph.numel() * 8)},
            "roofline": roof,
            "clocks": clk,
            "solver_ms_per_step": t_solve,
            "status_ok": int((status == 0).sum()), "status_total": int(status.size),
            "solver_counters": {"steps_mean": float(sts[:, 0].mean()), "rejected_mean": float(sts[:, 1].mean()),
                                "newton_iters_mean": float(sts[:, 2].mean()), "factorisations_mean": float(sts[:, 3].mean()),
                                "fp64_flops_per_step": flops},
        }
    ctx.close()
    if rank == 0 and world == 1:
        if not args.no_surrogate:
            out["surrogate"] = surrogate_leg(fp, dev)
        if not args.no_sweep:
            out["sweep"] = sweep_leg(fp, dev, args.sweep_instances)
        if not args.no_adjoint:
            out["adjoint"] = adjoint_leg(fp, dev, stages=args.adjoint_stages)
        if not args.no_models:
            out["models"] = models_leg(fp, dev, peak / 1e3, args.m1_dictionary, args.m2_tuples)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return out, dspec, inst


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        from paper_2106_08040_gb300 import workloads
        dspec, inst = workloads.system_matrix_workload()
        vals = []
        t_all = time.time()
        for k in range(args.warmup + args.steps):
            r = cpu_oracle_sample(dspec, inst, args.cpu_sample_s / 2)
            if k >= args.warmup:
                vals.append(r)
        wall = time.time() - t_all
        v = statistics.mean(x["value"] for x in vals)
        cb = dict(vals[-1])
        cb["value"] = v
        out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * wall / (args.warmup + args.steps),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "impl": "reference",
               "config": {"workload": "system_matrix_32x32_L16_lissajous", "instances_per_gpu": len(inst), "L": 16,
                          "periods_per_instance": 2, "samples_per_period": 1632},
               "cpu_baseline": cb,
               "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return 0
    out, dspec, inst = run_gpu(args)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_oracle_sample(dspec, inst, args.cpu_sample_s)
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())

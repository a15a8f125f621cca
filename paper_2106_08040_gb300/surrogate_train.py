"""Train the harmonic surrogate on solves of the method and measure its error against them.

    python -m paper_2106_08040_gb300.surrogate_train --train 32768 --holdout 1024 \
        --steps 60000 --out paper_2106_08040_gb300/data/surrogate_L16.npz

1. Draw instances from the uneven-sweep distribution (voxel offsets on the
   z = 0 plane of a 24 mm field of view with gradient diag(-1, -1, 2) T/m,
   16 Fibonacci easy-axis directions, K log-uniform 5e2..1e4 J/m^3, d
   log-normal around 20 nm) at truncation degree L, keeping the barriers
   sigma = K V / (k_B T) <= sigma_max that degree L resolves.
2. Solve each under the cosine Lissajous drive (1 warm-up + 1 output period)
   with fp_solve_batch and take phi_hat of the x and y channels with
   fp_signal: the training targets are harmonics k = 1..200.
3. Fit two networks (different seeds) with fp_surrogate_grad/fp_surrogate_adam.
   Their mean is the surrogate's answer and their disagreement its error
   estimate: queries whose estimate exceeds the gate go to the solver.
4. Report the held-out relative error of the mean against the solver.
"""
import argparse
import json
import os
import time

import numpy as np

from . import fp, surrogate, workloads

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "data", "surrogate_L16.npz")
K_MAX = surrogate.N_HARM


def solver_context(L, rtol, stages=3):
    dspec = workloads.drive_lissajous()
    return fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=rtol, stages=stages), L)


def solve_signals(ctx, inst, batch=2048):
    """Targets [n, 800] (phi_hat of channels x, y, k = 1..200) and status [n]
    for host instance records, solved on the current device in batches."""
    import torch
    n = len(inst)
    y = np.zeros((n, surrogate.N_OUT))
    status = np.zeros(n, dtype=np.int32)
    ch = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]
    for a in range(0, n, batch):
        sub = inst[a:a + batch]
        _, dm, st, _ = fp.solve(ctx, sub, want_m=False)
        ph = torch.empty((len(sub), 2, K_MAX + 1, 2), dtype=torch.float64, device=dm.device)
        fp.fp_signal(ctx, dm, len(sub), K_MAX, ch, ph)
        torch.cuda.synchronize()
        y[a:a + len(sub)] = surrogate.targets_from_phihat(ph.cpu().numpy())
        status[a:a + len(sub)] = st.cpu().numpy()
        del dm, ph
    return y, status


def relative_errors(y_hat, y):
    return np.linalg.norm(y_hat - y, axis=1) / np.linalg.norm(y, axis=1)


class Ensemble:
    """Two surrogates; answer = mean, error estimate = half their distance
    relative to the answer's norm."""

    def __init__(self, members):
        self.members = members

    def infer(self, x, stream=None):
        """Mean and spread in one pass (fp_surrogate_infer_ensemble)."""
        import ctypes as C
        import torch
        from . import _lib
        a, b = self.members
        q = x.shape[0]
        mean = torch.empty((q, surrogate.N_OUT), dtype=torch.float32, device=a.device)
        spread = torch.empty((q,), dtype=torch.float32, device=a.device)
        ws = a.workspace(q, 2)
        s = stream if stream is not None else torch.cuda.current_stream()
        _lib.check(_lib.lib().fp_surrogate_infer_ensemble(C.byref(a.net), C.byref(b.net), C.c_void_p(x.data_ptr()),
                                                          int(q), C.c_void_p(mean.data_ptr()),
                                                          C.c_void_p(spread.data_ptr()), C.c_void_p(ws.data_ptr()),
                                                          C.c_ulonglong(ws.numel()), C.c_void_p(a._err.data_ptr()),
                                                          C.c_void_p(s.cuda_stream)), "fp_surrogate_infer_ensemble")
        return mean, spread

    def save(self, path, **meta):
        base, ext = os.path.splitext(path)
        for i, m in enumerate(self.members):
            m.save("%s.m%d%s" % (base, i, ext), **meta)

    @classmethod
    def load(cls, path, device="cuda"):
        base, ext = os.path.splitext(path)
        return cls([surrogate.Surrogate.load("%s.m%d%s" % (base, i, ext), device=device) for i in range(2)])


def main():
    import torch
    p = argparse.ArgumentParser()
    p.add_argument("--train", type=int, default=32768)
    p.add_argument("--holdout", type=int, default=1024)
    p.add_argument("--L", type=int, default=16)
    p.add_argument("--rtol", type=float, default=1e-7)
    p.add_argument("--steps", type=int, default=60000)
    p.add_argument("--batch", type=int, default=4096)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--seed", type=int, default=workloads.SEED)
    p.add_argument("--sigma-max", type=float, default=12.0,
                   help="domain cap on K V / (k_B T): at L = 16 larger barriers are not resolved")
    p.add_argument("--out", default=DEFAULT_OUT)
    p.add_argument("--dump", default="", help="also write the solved dataset (npz) here")
    p.add_argument("--from-dump", default="", help="train on a dataset written by --dump instead of solving")
    a = p.parse_args()
    torch.cuda.set_device(0)
    # draw, keep the barriers degree L resolves, then split train / holdout
    draw = workloads.uneven_sweep_instances(2 * (a.train + a.holdout), a.L, seed=a.seed)
    in_domain = fp.Material().sigma(draw["K"], draw["d"]) <= a.sigma_max
    inst = draw[in_domain][:a.train + a.holdout]
    t0 = time.time()
    if a.from_dump:
        z = np.load(a.from_dump)
        y, st = z["y"].astype(np.float64), z["status"]
        assert len(y) == len(inst)
    else:
        ctx = solver_context(a.L, a.rtol)
        y, st = solve_signals(ctx, inst)
        ctx.close()
        if a.dump:
            np.savez_compressed(a.dump, y=y.astype(np.float32), status=st)
    t_solve = time.time() - t0
    x = surrogate.features(inst)
    ok = (st == 0) & np.all(np.isfinite(y), axis=1)
    tr = np.flatnonzero(ok[:a.train])
    ho = a.train + np.flatnonzero(ok[a.train:])
    print(json.dumps({"solved": int(len(inst)), "ok": int(ok.sum()), "in_domain_fraction": float(in_domain.mean()),
                      "status": np.bincount(st, minlength=7).tolist(), "solve_s": t_solve}), flush=True)
    members = []
    xt = torch.from_numpy(x[tr].astype(np.float32)).cuda()
    yt = torch.from_numpy(y[tr].astype(np.float32)).cuda()
    t0 = time.time()
    for s in range(2):
        m = surrogate.Surrogate(seed=a.seed + s)
        m.set_normalisation(x[tr], y[tr])
        hist = m.fit(xt, yt, a.steps, batch=a.batch, lr=a.lr, seed=s, log_every=max(1, a.steps // 10))
        torch.cuda.synchronize()
        print(json.dumps({"member": s, "loss": hist, "err_flag": m.error_flag()}), flush=True)
        members.append(m)
    t_fit = time.time() - t0
    ens = Ensemble(members)
    mean, spread = ens.infer(torch.from_numpy(x[ho].astype(np.float32)).cuda())
    err = relative_errors(mean.cpu().numpy().astype(np.float64), y[ho])
    spr = spread.cpu().numpy()
    rep = {"train": int(len(tr)), "holdout": int(len(ho)), "fit_s": t_fit, "solve_s": t_solve,
           "holdout_err_median": float(np.median(err)), "holdout_err_p90": float(np.quantile(err, 0.9)),
           "holdout_err_max": float(err.max()), "spread_median": float(np.median(spr)),
           "accepted_at_1e-3": float(np.mean(spr <= 1e-3)),
           "err_of_accepted_max": float(err[spr <= 1e-3].max()) if np.any(spr <= 1e-3) else None}
    print(json.dumps(rep), flush=True)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    ens.save(a.out, L=a.L, rtol=a.rtol, train=len(tr), steps=a.steps, seed=a.seed)


if __name__ == "__main__":
    main()

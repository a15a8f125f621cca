"""Adjoint-driven parameter fits on synthetic measurements.

The measurement over a voxel grid is a weighted superposition of the signals
of a few hidden parameter sets (K, d, theta, phi) plus Gaussian noise; a
candidate parameter set p explains it with the single-set model phi_hat(v; p)
at every voxel v (the superposition and single-function-vector models of
Sec. 2.2, M1, with the transfer function left out, R7).  The misfit

    J(p) = sum_v sum_{c, k} |phi_hat_{c,k}(v; p) - u_{c,k}(v)|^2

and its gradient dJ/d(K, d, theta, phi) come from one forward solve per voxel
(fp_solve_batch + fp_signal) and one adjoint per voxel (fp_grad with
dJ/dphi_hat = 2 (phi_hat - u)), summed over the voxels of each candidate.

The superposition model (the polydisperse model of Sec. 2.2, M2, with its
weights fitted together with the parameters) explains the measurement by
sum_j w_j phi_hat(v; p_j), w_j >= 0, for J parameter sets at once:

    J(p, w) = sum_v sum_{c, k} |sum_j w_j phi_hat_{c,k}(v; p_j) - u_{c,k}(v)|^2,
    dJ/dw_j = 2 <r, phi_hat(p_j)>,  dJ/dp_j = adjoint of phi_hat(.; p_j) with
    cotangent 2 w_j r  (r = model - u, real and imaginary parts as reals).
"""
import numpy as np

from . import fp, workloads


class FitProblem:
    def __init__(self, dspec, offsets, L, k_max, rtol=1e-9, channels=((1.0, 0.0, 0.0), (0.0, 1.0, 0.0))):
        self.dspec, self.offsets, self.L, self.k_max = dspec, np.asarray(offsets), L, k_max
        self.ch = np.asarray(channels, dtype=np.float64)
        self.ctx = fp.Context(fp.Material(), fp.Drive(**dspec.__dict__), fp.Tol(rtol=rtol, stages=3), L)

    def instances(self, params):
        """One instance per (candidate, voxel): params [P, 4] = (K, d, theta, phi)."""
        params = np.atleast_2d(params)
        nv = len(self.offsets)
        inst = workloads.make_instances(len(params) * nv)
        inst["h_off"] = np.tile(self.offsets, (len(params), 1))
        for j, key in enumerate(("K", "d", "theta", "phi")):
            inst[key] = np.repeat(params[:, j], nv)
        inst["L"] = self.L
        return inst

    def signals(self, params):
        """phi_hat [P, V, C, k_max + 1, 2] (device tensor) and status [P * V]."""
        import torch
        inst = self.instances(params)
        _, dm, st, _ = fp.solve(self.ctx, inst, want_m=False)
        ph = torch.empty((len(inst), len(self.ch), self.k_max + 1, 2), dtype=torch.float64, device=dm.device)
        fp.fp_signal(self.ctx, dm, len(inst), self.k_max, self.ch, ph)
        P = np.atleast_2d(params).shape[0]
        return ph.view(P, len(self.offsets), len(self.ch), self.k_max + 1, 2), st

    def measurement(self, hidden, weights, noise=0.01, seed=workloads.SEED):
        """sum_i w_i phi_hat(v; p_i) + Gaussian noise of `noise` x the RMS signal."""
        ph, st = self.signals(hidden)
        if not bool((st == 0).all()):
            raise RuntimeError("hidden parameter sets did not solve: %s" % st.cpu().numpy())
        import torch
        w = torch.as_tensor(np.asarray(weights, dtype=np.float64), device=ph.device).view(-1, 1, 1, 1, 1)
        u = (w * ph).sum(dim=0)
        rms = float(u.pow(2).mean().sqrt())
        g = torch.Generator(device=ph.device)
        g.manual_seed(int(seed))
        return u + noise * rms * torch.randn(u.shape, generator=g, device=u.device, dtype=u.dtype)

    def misfit_and_grad(self, params, u):
        """J [P] and dJ/d(K, d, theta, phi) [P, 4] for candidate sets params [P, 4]."""
        import torch
        params = np.atleast_2d(params)
        inst = self.instances(params)
        ph, st = self.signals(params)
        r = ph - u.unsqueeze(0)
        J = r.pow(2).sum(dim=(1, 2, 3, 4))
        n = len(inst)
        dev = ph.device
        d_inst = fp.instances_to_device(inst, dev)
        dJ = (2.0 * r).reshape(n, len(self.ch), self.k_max + 1, 2).contiguous()
        grad = torch.empty((n, 4), dtype=torch.float64, device=dev)
        gst = torch.empty((n,), dtype=torch.int32, device=dev)
        work = torch.empty(fp.fp_grad_workspace_bytes(self.ctx, n), dtype=torch.uint8, device=dev)
        fp.fp_grad(self.ctx, d_inst, n, self.k_max, self.ch, dJ, grad, gst, work)
        ok = bool((st == 0).all()) and bool((gst == 0).all())
        g = grad.view(len(params), len(self.offsets), 4).sum(dim=1)
        return J.cpu().numpy(), g.cpu().numpy(), ok

    def fit(self, params0, u, iters=20, lr=0.05, beta1=0.9, beta2=0.999):
        """Adam on q = (ln K, ln d, theta, phi) of each candidate, gradients by the
        adjoint (dJ/dln K = K dJ/dK, likewise d).  Returns the final parameters
        [P, 4] and the misfit history [iters + 1, P]."""
        p = np.atleast_2d(np.asarray(params0, dtype=np.float64)).copy()
        q = np.column_stack([np.log(p[:, 0]), np.log(p[:, 1]), p[:, 2], p[:, 3]])
        m = np.zeros_like(q)
        v = np.zeros_like(q)
        hist = []
        for it in range(iters + 1):
            p = np.column_stack([np.exp(q[:, 0]), np.exp(q[:, 1]), q[:, 2], q[:, 3]])
            J, g, ok = self.misfit_and_grad(p, u)
            if not ok:
                raise RuntimeError("solve or adjoint did not converge at iteration %d" % it)
            hist.append(J)
            if it == iters:
                break
            gq = g * np.column_stack([p[:, 0], p[:, 1], np.ones(len(p)), np.ones(len(p))])
            m = beta1 * m + (1 - beta1) * gq
            v = beta2 * v + (1 - beta2) * gq * gq
            mh = m / (1 - beta1 ** (it + 1))
            vh = v / (1 - beta2 ** (it + 1))
            q = q - lr * mh / (np.sqrt(vh) + 1e-30)
        return p, np.array(hist)

    def superposition_misfit_and_grad(self, params, weights, u):
        """J, dJ/d(K, d, theta, phi) [J, 4] and dJ/dw [J] of the superposition
        model sum_j w_j phi_hat(v; p_j) for parameter sets params [J, 4] and
        weights [J]."""
        import torch
        params = np.atleast_2d(params)
        nset, nv = len(params), len(self.offsets)
        inst = self.instances(params)
        ph, st = self.signals(params)                                  # [J, V, C, K, 2]
        w = torch.as_tensor(np.asarray(weights, dtype=np.float64), device=ph.device)
        r = (w.view(-1, 1, 1, 1, 1) * ph).sum(dim=0) - u               # [V, C, K, 2]
        J = float(r.pow(2).sum())
        gw = 2.0 * (ph * r.unsqueeze(0)).sum(dim=(1, 2, 3, 4))
        n = len(inst)
        dev = ph.device
        dJ = (2.0 * w.view(-1, 1, 1, 1, 1) * r.unsqueeze(0)).reshape(n, len(self.ch), self.k_max + 1, 2).contiguous()
        grad = torch.empty((n, 4), dtype=torch.float64, device=dev)
        gst = torch.empty((n,), dtype=torch.int32, device=dev)
        work = torch.empty(fp.fp_grad_workspace_bytes(self.ctx, n), dtype=torch.uint8, device=dev)
        fp.fp_grad(self.ctx, fp.instances_to_device(inst, dev), n, self.k_max, self.ch, dJ, grad, gst, work)
        ok = bool((st == 0).all()) and bool((gst == 0).all())
        g = grad.view(nset, nv, 4).sum(dim=1)
        return J, g.cpu().numpy(), gw.cpu().numpy(), ok

    def fit_superposition(self, params0, weights0, u, iters=20, lr=0.05, beta1=0.9, beta2=0.999):
        """Adam on (ln K, ln d, theta, phi, ln w) of every set (w = exp(.) keeps
        the weights non-negative), gradients by the adjoint.  Returns the final
        parameters [J, 4], weights [J] and the misfit history [iters + 1]."""
        p = np.atleast_2d(np.asarray(params0, dtype=np.float64)).copy()
        q = np.column_stack([np.log(p[:, 0]), np.log(p[:, 1]), p[:, 2], p[:, 3],
                             np.log(np.asarray(weights0, dtype=np.float64))])
        m = np.zeros_like(q)
        v = np.zeros_like(q)
        hist = []
        for it in range(iters + 1):
            p = np.column_stack([np.exp(q[:, 0]), np.exp(q[:, 1]), q[:, 2], q[:, 3]])
            w = np.exp(q[:, 4])
            J, g, gw, ok = self.superposition_misfit_and_grad(p, w, u)
            if not ok:
                raise RuntimeError("solve or adjoint did not converge at iteration %d" % it)
            hist.append(J)
            if it == iters:
                break
            gq = np.column_stack([g[:, 0] * p[:, 0], g[:, 1] * p[:, 1], g[:, 2], g[:, 3], gw * w])
            m = beta1 * m + (1 - beta1) * gq
            v = beta2 * v + (1 - beta2) * gq * gq
            mh = m / (1 - beta1 ** (it + 1))
            vh = v / (1 - beta2 ** (it + 1))
            q = q - lr * mh / (np.sqrt(vh) + 1e-30)
        return p, w, np.array(hist)

    def close(self):
        self.ctx.close()

"""Harmonic surrogate over libfp.so's tensor-core MLP kernels.

A multilayer perceptron 7 -> 512 -> 512 -> 512 -> 512 -> 800 (exact GELU)
maps one instance -- offset field B_off [T] (3), easy-axis theta, phi [rad],
ln K, ln d -- to the first 200 complex harmonics (k = 1..200) of the normalised
signal phi_hat of the x and y receive channels (Sec. 2.2, model M1), laid out
[channel][k-1][re, im].  The paper has no surrogate: the Fokker-Planck solve
produces its training data and is the reference for its error (and its fallback).

This module holds the weights (FP32 masters, BF16 copies, Adam moments) in
torch device tensors and marshals them to fp_surrogate_infer /
fp_surrogate_grad / fp_surrogate_adam; every arithmetic step of inference and
training runs in those kernels.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import check

K_IN, N_IN, HIDDEN, N_OUT, LAYERS = 64, 7, 512, 800, 5
KL = [K_IN, HIDDEN, HIDDEN, HIDDEN, HIDDEN]
NL = [HIDDEN, HIDDEN, HIDDEN, HIDDEN, N_OUT]
N_HARM = 200


def _p(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def features(inst):
    """Surrogate inputs [n, 7] from instance records: B_off (3), theta, phi, ln K, ln d."""
    x = np.empty((len(inst), N_IN), dtype=np.float64)
    x[:, 0:3] = inst["h_off"]
    x[:, 3] = inst["theta"]
    x[:, 4] = inst["phi"]
    x[:, 5] = np.log(inst["K"])
    x[:, 6] = np.log(inst["d"])
    return x


def targets_from_phihat(ph):
    """[n, 2, >=201, 2] phi_hat (k = 0..) -> [n, 800] targets (k = 1..200)."""
    return np.ascontiguousarray(ph[:, :, 1:N_HARM + 1, :]).reshape(len(ph), N_OUT)


class Surrogate:
    """Weights and optimiser state of the surrogate on one CUDA device."""

    def __init__(self, device="cuda", seed=0):
        import torch
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        f32 = dict(dtype=torch.float32, device=self.device)
        self.Wm, self.bm = [], []
        for l in range(LAYERS):
            w = np.zeros((NL[l], KL[l]), dtype=np.float32)
            k_eff = N_IN if l == 0 else KL[l]
            w[:, :k_eff] = rng.normal(0.0, 1.0 / np.sqrt(k_eff), size=(NL[l], k_eff))
            self.Wm.append(torch.from_numpy(w).to(self.device))
            self.bm.append(torch.zeros(NL[l], **f32))
        self.W = [torch.empty((NL[l], KL[l]), dtype=torch.bfloat16, device=self.device) for l in range(LAYERS)]
        self.WT = [torch.empty((KL[l], NL[l]), dtype=torch.bfloat16, device=self.device) for l in range(LAYERS)]
        self.mW = [torch.zeros_like(w) for w in self.Wm]
        self.vW = [torch.zeros_like(w) for w in self.Wm]
        self.mb = [torch.zeros_like(b) for b in self.bm]
        self.vb = [torch.zeros_like(b) for b in self.bm]
        self.gW = [torch.zeros_like(w) for w in self.Wm]
        self.gb = [torch.zeros_like(b) for b in self.bm]
        self.in_shift = torch.zeros(N_IN, **f32)
        self.in_scale = torch.ones(N_IN, **f32)
        self.out_shift = torch.zeros(N_OUT, **f32)
        self.out_scale = torch.ones(N_OUT, **f32)
        self.step = 0
        self._ws = {}
        self._err = torch.zeros(1, dtype=torch.int32, device=self.device)
        self._loss = torch.zeros(1, **f32)
        self._build_structs()
        self.refresh()

    # -------------------------------------------------------------- structs --
    def _build_structs(self):
        n = _lib.fp_surrogate()
        for l in range(LAYERS):
            n.W[l] = self.W[l].data_ptr()
            n.b[l] = self.bm[l].data_ptr()
        n.in_shift, n.in_scale = self.in_shift.data_ptr(), self.in_scale.data_ptr()
        n.out_shift, n.out_scale = self.out_shift.data_ptr(), self.out_scale.data_ptr()
        t = _lib.fp_surrogate_train()
        t.net = n
        for l in range(LAYERS):
            t.WT[l] = self.WT[l].data_ptr()
            t.Wm[l] = self.Wm[l].data_ptr()
            t.bm[l] = self.bm[l].data_ptr()
            t.mW[l], t.vW[l] = self.mW[l].data_ptr(), self.vW[l].data_ptr()
            t.mb[l], t.vb[l] = self.mb[l].data_ptr(), self.vb[l].data_ptr()
        self.net, self.train_state = n, t
        self._gW = (C.c_void_p * LAYERS)(*[g.data_ptr() for g in self.gW])
        self._gb = (C.c_void_p * LAYERS)(*[g.data_ptr() for g in self.gb])

    def refresh(self, stream=None):
        """Rewrite the BF16 copies (W, W^T) from the FP32 masters."""
        check(_lib.lib().fp_surrogate_adam(C.byref(self.train_state), None, None, 0.0, 0.9, 0.999, 1e-8, 0,
                                           _stream(stream)), "fp_surrogate_adam")

    def set_normalisation(self, x, y, per_output=False):
        """Input shift/scale and output shift/scale from training data (host
        arrays).  By default the outputs share one scale (the RMS deviation of
        all of them), so the squared-error loss weighs each harmonic as the
        relative L2 signal error does; per_output=True standardises each
        output column instead."""
        import torch
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        xs = x.std(axis=0)
        self.in_shift.copy_(torch.from_numpy(x.mean(axis=0).astype(np.float32)))
        self.in_scale.copy_(torch.from_numpy((1.0 / np.where(xs > 0, xs, 1.0)).astype(np.float32)))
        mu = y.mean(axis=0)
        self.out_shift.copy_(torch.from_numpy(mu.astype(np.float32)))
        if per_output:
            ys = y.std(axis=0)
            ys = np.maximum(ys, 1e-3 * max(float(ys.max()), 1e-30))
        else:
            ys = np.full(y.shape[1], max(float(np.sqrt(np.mean((y - mu) ** 2))), 1e-30))
        self.out_scale.copy_(torch.from_numpy(ys.astype(np.float32)))

    def workspace(self, q, training):
        import torch
        key = (q, training)
        if key not in self._ws:
            nb = _lib.lib().fp_surrogate_workspace_bytes(int(q), int(training))
            if nb < 0:
                check(int(nb), "fp_surrogate_workspace_bytes")
            self._ws[key] = torch.empty(int(nb), dtype=torch.uint8, device=self.device)
        return self._ws[key]

    # ----------------------------------------------------------- inference --
    def infer(self, x, out=None, stream=None):
        """x: device f32 [q, 7] -> device f32 [q, 800]."""
        import torch
        q = x.shape[0]
        y = out if out is not None else torch.empty((q, N_OUT), dtype=torch.float32, device=self.device)
        ws = self.workspace(q, 0)
        check(_lib.lib().fp_surrogate_infer(C.byref(self.net), _p(x), int(q), _p(y), _p(ws), C.c_ulonglong(ws.numel()),
                                            _p(self._err), _stream(stream)), "fp_surrogate_infer")
        return y

    # ------------------------------------------------------------ training --
    def grad(self, x, y, stream=None):
        """Loss (sum of squared normalised errors) into self._loss, gradients into self.gW/gb."""
        q = x.shape[0]
        ws = self.workspace(q, 1)
        check(_lib.lib().fp_surrogate_grad(C.byref(self.train_state), _p(x), _p(y), int(q), _p(self._loss),
                                           self._gW, self._gb, _p(ws), C.c_ulonglong(ws.numel()), _p(self._err),
                                           _stream(stream)), "fp_surrogate_grad")
        return self._loss

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.step += 1
        check(_lib.lib().fp_surrogate_adam(C.byref(self.train_state), self._gW, self._gb, float(lr), float(beta1),
                                           float(beta2), float(eps), int(self.step), _stream(stream)),
              "fp_surrogate_adam")

    def fit(self, x, y, steps, batch=4096, lr=1e-3, lr_min=1e-5, seed=0, log_every=0):
        """Adam on random minibatches of device tensors x [n, 7], y [n, 800];
        cosine learning-rate decay from lr to lr_min.  Returns the loss history
        (mean squared normalised error per logged step)."""
        import torch
        n = x.shape[0]
        batch = min(batch, n - n % 8)
        g = torch.Generator(device=self.device)
        g.manual_seed(seed)
        hist = []
        for s in range(steps):
            idx = torch.randint(0, n, (batch,), generator=g, device=self.device)
            self.grad(x[idx].contiguous(), y[idx].contiguous())
            lr_s = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * s / max(steps, 1)))
            self.adam(lr_s)
            if log_every and (s % log_every == 0 or s == steps - 1):
                hist.append((s, float(self._loss.item()) / (batch * N_OUT)))
        return hist

    def error_flag(self):
        return int(self._err.item())

    # ------------------------------------------------------------- storage --
    def state(self):
        return {"Wm": [w.cpu().numpy() for w in self.Wm], "bm": [b.cpu().numpy() for b in self.bm],
                "in_shift": self.in_shift.cpu().numpy(), "in_scale": self.in_scale.cpu().numpy(),
                "out_shift": self.out_shift.cpu().numpy(), "out_scale": self.out_scale.cpu().numpy()}

    def save(self, path, **meta):
        """Weights as their BF16 bit patterns (what inference uses), the rest in FP32."""
        s = self.state()
        arrs = {"W%d" % l: self.W[l].cpu().view(__import__("torch").int16).numpy() for l in range(LAYERS)}
        arrs.update({"b%d" % l: s["bm"][l] for l in range(LAYERS)})
        arrs.update({k: s[k] for k in ("in_shift", "in_scale", "out_shift", "out_scale")})
        arrs.update({"meta_" + k: np.asarray(v) for k, v in meta.items()})
        np.savez_compressed(path, **arrs)

    @classmethod
    def load(cls, path, device="cuda"):
        import torch
        z = np.load(path)
        s = cls(device=device)
        for l in range(LAYERS):
            w = z["W%d" % l]
            if w.dtype == np.int16:
                w = torch.from_numpy(w).view(torch.bfloat16).float()
            else:
                w = torch.from_numpy(w)
            s.Wm[l].copy_(w)
            s.bm[l].copy_(torch.from_numpy(z["b%d" % l]))
        for k in ("in_shift", "in_scale", "out_shift", "out_scale"):
            getattr(s, k).copy_(torch.from_numpy(z[k]))
        s.refresh()
        return s


def main():
    """Time inference of an untrained network (random weights, random inputs):
    python -m paper_2106_08040_gb300.surrogate --queries 1024000 --repeat 10"""
    import argparse
    import json
    import torch
    p = argparse.ArgumentParser()
    p.add_argument("--queries", type=int, default=1024000)
    p.add_argument("--repeat", type=int, default=10)
    p.add_argument("--seed", type=int, default=1)
    a = p.parse_args()
    s = Surrogate(seed=a.seed)
    g = torch.Generator(device="cuda")
    g.manual_seed(a.seed)
    x = torch.randn(a.queries, N_IN, device="cuda", generator=g)
    y = torch.empty(a.queries, N_OUT, device="cuda")
    s.infer(x, out=y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.repeat):
        s.infer(x, out=y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.repeat, 1)
    flops = 2.0 * a.queries * (N_IN * HIDDEN + 3 * HIDDEN * HIDDEN + HIDDEN * N_OUT)
    print(json.dumps({"queries": a.queries, "ms_per_network": ms, "tflops_algorithmic": flops / (ms * 1e-3) / 1e12,
                      "err_flag": s.error_flag()}))


if __name__ == "__main__":
    main()

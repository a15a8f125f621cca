"""Python binding of libfp.so with the C-ABI names (include/fp.h).

Argument marshalling only: every step of the solve runs in the CUDA kernels.
Device buffers are torch CUDA tensors (torch supplies memory and streams).
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import check, fp_drive, fp_instance, fp_material, fp_tol

INSTANCE_DTYPE = np.dtype([("h_off", "<f8", (3,)), ("theta", "<f8"), ("phi", "<f8"), ("K", "<f8"),
                           ("d", "<f8"), ("L", "<i4"), ("flags", "<i4")])
assert INSTANCE_DTYPE.itemsize == 64


@dataclass(frozen=True)
class Material:
    """Sec. 2.1 material constants (SI)."""
    Ms: float = 474e3
    alpha: float = 0.1
    gamma: float = 1.76e11
    T_B: float = 293.0

    def c(self):
        return fp_material(self.Ms, self.alpha, self.gamma, self.T_B)

    def sigma(self, K, d):
        """Anisotropy barrier sigma = K V / (k_B T), V = pi d^3 / 6 (Sec. 2.1)."""
        return np.asarray(K) * np.pi * np.asarray(d) ** 3 / 6.0 / (1.380649e-23 * self.T_B)


@dataclass(frozen=True)
class Drive:
    """B_k(t) = amp_k sin(2 pi freq_k t + phase_k) [T]; sampling schedule."""
    amp: tuple
    freq: tuple
    phase: tuple
    period: float
    samples_per_period: int
    warmup_periods: int
    output_periods: int

    def c(self):
        d = fp_drive()
        for k in range(3):
            d.amp[k], d.freq[k], d.phase[k] = self.amp[k], self.freq[k], self.phase[k]
        d.period = self.period
        d.samples_per_period = self.samples_per_period
        d.warmup_periods = self.warmup_periods
        d.output_periods = self.output_periods
        return d

    @property
    def num_samples(self):
        return self.output_periods * self.samples_per_period


@dataclass(frozen=True)
class Tol:
    rtol: float = 1e-9
    atol: float = 1e-15
    max_steps: int = 2_000_000
    newton_max_iter: int = 8
    refactor_every: int = 8
    checkpoint_every: int = 64
    stages: int = 5

    def c(self):
        return fp_tol(self.rtol, self.atol, self.max_steps, self.newton_max_iter,
                      self.refactor_every, self.checkpoint_every, self.stages, 0)


def fp_peak_fp64():
    """Measured FP64 FMA throughput of the current device [GFLOP/s]."""
    v = C.c_double()
    check(_lib.lib().fp_peak_fp64(C.byref(v)), "fp_peak_fp64")
    return v.value


def fp_max_degree():
    return _lib.lib().fp_max_degree()


class Context:
    """Owns an fp_ctx (coefficient tables on the current CUDA device)."""

    def __init__(self, material: Material, drive: Drive, tol: Tol, L_max: int):
        self.material, self.drive, self.tol, self.L_max = material, drive, tol, L_max
        h = C.c_void_p()
        m, d, t = material.c(), drive.c(), tol.c()
        check(_lib.lib().fp_setup(C.byref(m), C.byref(d), C.byref(t), int(L_max), C.byref(h)), "fp_setup")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("context destroyed")
        return self._h

    def num_samples(self):
        return _lib.lib().fp_num_samples(self.handle)

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.lib().fp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp_setup(material: Material, drive: Drive, tol: Tol, L_max: int) -> Context:
    return Context(material, drive, tol, L_max)


def fp_destroy(ctx: Context):
    ctx.close()


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def instances_to_device(inst: np.ndarray, device="cuda"):
    """Pack a structured INSTANCE_DTYPE array into a device byte tensor."""
    import torch
    arr = np.ascontiguousarray(inst, dtype=INSTANCE_DTYPE)
    host = torch.from_numpy(arr.view(np.uint8).reshape(-1).copy())
    return host.to(device)


def fp_solve_batch(ctx: Context, d_inst, n: int, d_m=None, d_dmdt=None, d_status=None, d_stats=None, stream=None):
    """Launch the batched solve; buffers are torch CUDA tensors (float64 [n,S,3],
    int32 [n], int32 [n,4])."""
    check(_lib.lib().fp_solve_batch(ctx.handle, _ptr(d_inst), int(n), _ptr(d_m), _ptr(d_dmdt), _ptr(d_status),
                                    _ptr(d_stats), _stream_ptr(stream)), "fp_solve_batch")


def fp_signal(ctx: Context, d_dmdt, n: int, k_max: int, channels, d_phihat, stream=None):
    ch = np.ascontiguousarray(np.asarray(channels, dtype=np.float64).reshape(-1, 3))
    check(_lib.lib().fp_signal(ctx.handle, _ptr(d_dmdt), int(n), int(k_max),
                               ch.ctypes.data_as(C.POINTER(C.c_double)), int(ch.shape[0]), _ptr(d_phihat),
                               _stream_ptr(stream)), "fp_signal")


def fp_equilibrium(ctx: Context, d_inst, n: int, d_m=None, d_dmdt=None, stream=None):
    """Model M0 traces (Sec. 2.2, Eq. Langevin) in the layouts of fp_solve_batch."""
    check(_lib.lib().fp_equilibrium(ctx.handle, _ptr(d_inst), int(n), _ptr(d_m), _ptr(d_dmdt), _stream_ptr(stream)),
          "fp_equilibrium")


def fp_m1_fit(d_phi, Q: int, d_S, N: int, C: int, K1: int, d_a, d_eps, d_smax, stream=None):
    """Model M1 fit per dictionary element, channel and row (Sec. 2.2) and the
    row errors of Eq. error1."""
    check(_lib.lib().fp_m1_fit(_ptr(d_phi), int(Q), _ptr(d_S), int(N), int(C), int(K1), _ptr(d_a), _ptr(d_eps),
                               _ptr(d_smax), _stream_ptr(stream)), "fp_m1_fit")


def fp_nrmse(d_eps, A: int, C: int, K1: int, d_ks, nk: int, d_eps_freq, d_eps_global, stream=None):
    """Per-frequency and global NRMSE (Sec. 2.3)."""
    check(_lib.lib().fp_nrmse(_ptr(d_eps), int(A), int(C), int(K1), _ptr(d_ks), int(nk), _ptr(d_eps_freq),
                              _ptr(d_eps_global), _stream_ptr(stream)), "fp_nrmse")


def fp_mixing_order(k: int, n_dens: int):
    """(m_x, m_y) of frequency index k (Eq. mix)."""
    mx, my = C.c_int(), C.c_int()
    check(_lib.lib().fp_mixing_order(int(k), int(n_dens), C.byref(mx), C.byref(my)), "fp_mixing_order")
    return mx.value, my.value


def fp_freq_index_set(M_x: int, M_y: int, n_dens: int, k_limit: int):
    """I_freq of Sec. 2.3 as a numpy int32 array."""
    cnt = C.c_int()
    check(_lib.lib().fp_freq_index_set(int(M_x), int(M_y), int(n_dens), int(k_limit), None, 0, C.byref(cnt)),
          "fp_freq_index_set")
    out = np.zeros(max(cnt.value, 1), dtype=np.int32)
    check(_lib.lib().fp_freq_index_set(int(M_x), int(M_y), int(n_dens), int(k_limit),
                                       out.ctypes.data_as(C.POINTER(C.c_int)), int(out.size), C.byref(cnt)),
          "fp_freq_index_set")
    return out[:cnt.value]


def fp_m2_gram(d_phi, d_a, d_S, d_smax, A: int, J: int, N: int, C_: int, K1: int, d_ks, nk: int, d_G, stream=None):
    """Complex Gram matrix of the Sigma-weighted M2 dictionary augmented with the data (Sec. 2.2)."""
    check(_lib.lib().fp_m2_gram(_ptr(d_phi), _ptr(d_a), _ptr(d_S), _ptr(d_smax), int(A), int(J), int(N), int(C_),
                                int(K1), _ptr(d_ks), int(nk), _ptr(d_G), _stream_ptr(stream)), "fp_m2_gram")


def fp_m2_solve(G, J: int, s_rank: int = 0):
    """M2 weights w >= 0 from a host Gram matrix [(J+1),(J+1),2]: (w, truncated
    objective, ||M w - y||^2, singular values, rank used)."""
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64))
    w = np.zeros(J)
    sv = np.zeros(J)
    obj, res = C.c_double(), C.c_double()
    dp = C.POINTER(C.c_double)
    rc = _lib.lib().fp_m2_solve(G.ctypes.data_as(dp), int(J), int(s_rank), w.ctypes.data_as(dp), C.byref(obj),
                                C.byref(res), sv.ctypes.data_as(dp))
    if rc < 0:
        check(rc, "fp_m2_solve")
    return w, obj.value, res.value, sv, rc


def fp_grad_workspace_bytes(ctx: Context, n: int) -> int:
    v = _lib.lib().fp_grad_workspace_bytes(ctx.handle, int(n))
    if v < 0:
        check(int(v), "fp_grad_workspace_bytes")
    return int(v)


def fp_grad(ctx: Context, d_inst, n: int, k_max: int, channels, d_dJ, d_grad, d_status, d_work, d_stats=None,
            stream=None):
    """Discrete adjoint: d_grad[n,4] = dJ/d(K, d, theta, phi) given dJ/dphi_hat."""
    ch = np.ascontiguousarray(np.asarray(channels, dtype=np.float64).reshape(-1, 3))
    nbytes = d_work.numel() * d_work.element_size()
    check(_lib.lib().fp_grad(ctx.handle, _ptr(d_inst), int(n), int(k_max),
                             ch.ctypes.data_as(C.POINTER(C.c_double)), int(ch.shape[0]), _ptr(d_dJ), _ptr(d_grad),
                             _ptr(d_status), _ptr(d_stats), _ptr(d_work), C.c_ulonglong(nbytes),
                             _stream_ptr(stream)), "fp_grad")


def fp_grad_noalloc(ctx: Context, d_inst, n: int, k_max: int, channels, d_dJ, d_grad, d_status, d_stats=None,
                    stream=None):
    """fp_grad on the library's fixed device scratch array: no workspace and
    no device allocation, for callers that may not allocate device memory when
    they call.  Calls whose launches may overlap on the GPU share the array and
    race; the first call on a device should come before any stream capture."""
    ch = np.ascontiguousarray(np.asarray(channels, dtype=np.float64).reshape(-1, 3))
    check(_lib.lib().fp_grad_noalloc(ctx.handle, _ptr(d_inst), int(n), int(k_max),
                                     ch.ctypes.data_as(C.POINTER(C.c_double)), int(ch.shape[0]), _ptr(d_dJ),
                                     _ptr(d_grad), _ptr(d_status), _ptr(d_stats), _stream_ptr(stream)),
          "fp_grad_noalloc")


def pack_instances(h_off, params, L, device):
    """Device instance records from tensors: h_off [n,3], params [n,4] =
    (K, d, theta, phi), L int.  Float64 columns + (L, flags) int32 pair."""
    import torch
    n = params.shape[0]
    Lf = torch.zeros((n, 2), dtype=torch.int32, device=device)
    Lf[:, 0] = L
    cols = torch.cat([h_off.to(device, torch.float64), params[:, 2:4].to(device, torch.float64),
                      params[:, 0:2].to(device, torch.float64), Lf.view(torch.float64)], dim=1)
    return cols.contiguous().view(torch.uint8).reshape(-1)


def _autograd_function():
    import torch

    class PhiHat(torch.autograd.Function):
        """phi_hat [n, C, k_max+1, 2] of the batched solve as a function of the
        per-instance parameters (K, d, theta, phi); backward = fp_grad."""

        @staticmethod
        def forward(ctx_, params, h_off, fpctx, L, k_max, channels):
            dev = params.device
            n = params.shape[0]
            S = fpctx.num_samples()
            d_inst = pack_instances(h_off, params.detach(), L, dev)
            dm = torch.empty((n, S, 3), dtype=torch.float64, device=dev)
            st = torch.empty((n,), dtype=torch.int32, device=dev)
            fp_solve_batch(fpctx, d_inst, n, None, dm, st, None)
            ch = np.asarray(channels, dtype=np.float64).reshape(-1, 3)
            out = torch.empty((n, ch.shape[0], k_max + 1, 2), dtype=torch.float64, device=dev)
            fp_signal(fpctx, dm, n, k_max, ch, out)
            _raise_on_status(st, "solve")
            ctx_.save_for_backward(params.detach(), h_off)
            ctx_.fpctx, ctx_.L, ctx_.k_max, ctx_.ch = fpctx, L, k_max, ch
            ctx_.status = st
            return out

        @staticmethod
        def backward(ctx_, g):
            params, h_off = ctx_.saved_tensors
            dev = params.device
            n = params.shape[0]
            d_inst = pack_instances(h_off, params, ctx_.L, dev)
            grad = torch.empty((n, 4), dtype=torch.float64, device=dev)
            st = torch.empty((n,), dtype=torch.int32, device=dev)
            work = torch.empty(fp_grad_workspace_bytes(ctx_.fpctx, n), dtype=torch.uint8, device=dev)
            fp_grad(ctx_.fpctx, d_inst, n, ctx_.k_max, ctx_.ch, g.contiguous().to(torch.float64), grad, st, work)
            _raise_on_status(st, "adjoint")
            return grad.to(params.dtype), None, None, None, None, None

    return PhiHat


_PHIHAT = None


def _raise_on_status(st, what):
    """Fail loudly when any instance of an autograd pass did not converge."""
    s = st.cpu().numpy()
    if (s != 0).any():
        bad = {_lib.STATUS.get(int(v), str(int(v))): int((s == v).sum()) for v in np.unique(s[s != 0])}
        raise RuntimeError("phi_hat %s: %d of %d instances did not converge %s" % (what, int((s != 0).sum()), len(s), bad))


def phi_hat(params, h_off, fpctx, L, k_max, channels):
    """Differentiable phi_hat (torch.autograd) of the batched solve: params
    [n, 4] = (K, d, theta, phi), h_off [n, 3]; the backward pass is fp_grad
    (discrete adjoint).  Raises if any instance of either pass does not
    converge.  At L = 16 the adjoint needs a 3-stage context (a 5-stage one
    exceeds the shared memory of a CTA)."""
    global _PHIHAT
    if _PHIHAT is None:
        _PHIHAT = _autograd_function()
    return _PHIHAT.apply(params, h_off, fpctx, L, k_max, channels)


def fp_operator_dense(material: Material, L: int, K: float, d: float, B_nframe):
    """Dense easy-axis-frame Galerkin matrix (host only, no GPU)."""
    N = (L + 1) ** 2
    out = np.zeros((N, N))
    inst = fp_instance()
    inst.L, inst.K, inst.d = int(L), float(K), float(d)
    B = (C.c_double * 3)(*[float(x) for x in B_nframe])
    m = material.c()
    check(_lib.lib().fp_operator_dense(C.byref(m), C.byref(inst), B, out.ctypes.data_as(C.POINTER(C.c_double))),
          "fp_operator_dense")
    return out


def solve(ctx: Context, inst: np.ndarray, want_m=True, want_dmdt=True, stream=None):
    """Convenience: solve host instance records on the current device.
    Returns torch tensors (m, dmdt, status, stats) on the device."""
    import torch
    n = len(inst)
    S = ctx.num_samples()
    dev = torch.device("cuda", torch.cuda.current_device())
    d_inst = instances_to_device(inst, dev)
    m = torch.empty((n, S, 3), dtype=torch.float64, device=dev) if want_m else None
    dm = torch.empty((n, S, 3), dtype=torch.float64, device=dev) if want_dmdt else None
    st = torch.empty((n,), dtype=torch.int32, device=dev)
    stats = torch.empty((n, 4), dtype=torch.int32, device=dev)
    fp_solve_batch(ctx, d_inst, n, m, dm, st, stats, stream=stream)
    return m, dm, st, stats


def truncation_degree(inst, material=None, drive=None, L_min=8, L_max=16):
    """Per-instance truncation degree (fp_truncation_degree of the C ABI):
    L = clamp(L_min, L_max, ceil(2 + 5.5 sqrt(sigma + xi_max)))."""
    material = material or Material()
    if drive is None:
        drive = Drive(amp=(0.0, 0.0, 0.0), freq=(0.0, 0.0, 0.0), phase=(0.0, 0.0, 0.0), period=1.0,
                      samples_per_period=2, warmup_periods=0, output_periods=1)
    rec = np.ascontiguousarray(np.asarray(inst).astype(INSTANCE_DTYPE))
    out = np.zeros(max(len(rec), 1), dtype=np.int32)
    mat, drv = material.c(), drive.c()
    check(_lib.lib().fp_truncation_degree(C.byref(mat), C.byref(drv), rec.ctypes.data_as(C.c_void_p), len(rec),
                                          int(L_min), int(L_max), out.ctypes.data_as(C.POINTER(C.c_int))),
          "fp_truncation_degree")
    return out[:len(rec)].astype(int)


def sweep_order(inst: np.ndarray, material: Material, drive: Drive, L_max: int, bucket_width=1):
    """Host-only planning of a sweep (no GPU): queue order [n] and the buckets'
    (launch degree, size) list, as fp_sweep_plan computes them."""
    arr = np.ascontiguousarray(inst, dtype=INSTANCE_DTYPE)
    n = len(arr)
    order = np.zeros(n, dtype=np.int32)
    bL = (C.c_int * 64)()
    bc = (C.c_int * 64)()
    nb = C.c_int()
    m, d = material.c(), drive.c()
    check(_lib.lib().fp_sweep_order(C.byref(m), C.byref(d), int(L_max), arr.ctypes.data_as(C.c_void_p), n,
                                    int(bucket_width), order.ctypes.data_as(C.POINTER(C.c_int)), bL, bc,
                                    C.byref(nb)), "fp_sweep_order")
    return order, [(bL[k], bc[k]) for k in range(nb.value)]


class Sweep:
    """fp_sweep plan over host instance records (see include/fp.h)."""

    def __init__(self, ctx: Context, inst: np.ndarray, bucket_width=1):
        self.ctx = ctx
        arr = np.ascontiguousarray(inst, dtype=INSTANCE_DTYPE)
        self.n = len(arr)
        h = C.c_void_p()
        check(_lib.lib().fp_sweep_plan(ctx.handle, arr.ctypes.data_as(C.c_void_p), self.n, int(bucket_width),
                                       C.byref(h)), "fp_sweep_plan")
        self._h = h

    def run(self, d_inst, d_m, d_dmdt, d_status, d_stats=None, stream=None):
        check(_lib.lib().fp_sweep_run(self._h, _ptr(d_inst), _ptr(d_m), _ptr(d_dmdt), _ptr(d_status), _ptr(d_stats),
                                      _stream_ptr(stream)), "fp_sweep_run")

    def autotune(self, d_inst, d_m, d_dmdt, d_status, sample=64, stream=None):
        check(_lib.lib().fp_sweep_autotune(self._h, _ptr(d_inst), _ptr(d_m), _ptr(d_dmdt), _ptr(d_status),
                                           int(sample), _stream_ptr(stream)), "fp_sweep_autotune")

    def info(self):
        nb = C.c_int()
        arrs = [(C.c_int * 64)() for _ in range(4)]
        ms = (C.c_float * 64)()
        check(_lib.lib().fp_sweep_info(self._h, C.byref(nb), *arrs, ms), "fp_sweep_info")
        k = nb.value
        return [{"L": arrs[0][i], "count": arrs[1][i], "stages": arrs[2][i], "refactor_every": arrs[3][i],
                 "tuned_ms": ms[i]} for i in range(k)]

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.lib().fp_sweep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

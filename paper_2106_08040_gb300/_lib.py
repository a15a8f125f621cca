"""ctypes view of libfp.so (include/fp.h).  Argument marshalling only.

The library is loaded from this package directory; a missing or unloadable
library raises immediately -- there is no fallback implementation.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfp.so")

FP_OK, FP_EINVAL, FP_ECUDA, FP_ENOMEM, FP_EUNSUPPORTED = 0, -1, -2, -3, -4
STATUS = {0: "OK", 1: "MAXSTEPS", 2: "STEP_UNDERFLOW", 3: "NONFINITE", 4: "NEWTON_FAIL", 5: "BAD_INPUT",
          6: "UNRESOLVED"}

EXPORTED = ["fp_max_degree", "fp_setup", "fp_destroy", "fp_num_samples", "fp_solve_batch",
            "fp_signal", "fp_grad_workspace_bytes", "fp_grad", "fp_grad_noalloc", "fp_surrogate_workspace_bytes", "fp_surrogate_infer",
            "fp_surrogate_grad", "fp_surrogate_adam", "fp_sweep_plan", "fp_sweep_order", "fp_sweep_run",
            "fp_sweep_autotune", "fp_sweep_info", "fp_sweep_destroy", "fp_operator_dense", "fp_peak_fp64",
            "fp_status_str", "fp_last_error", "fp_equilibrium", "fp_m1_fit", "fp_nrmse", "fp_mixing_order",
            "fp_freq_index_set", "fp_truncation_degree", "fp_m2_gram_bytes", "fp_m2_gram", "fp_m2_solve", "fp_surrogate_infer_ensemble"]


class fp_material(C.Structure):
    _fields_ = [("Ms", C.c_double), ("alpha", C.c_double), ("gamma", C.c_double), ("T_B", C.c_double)]


class fp_drive(C.Structure):
    _fields_ = [("amp", C.c_double * 3), ("freq", C.c_double * 3), ("phase", C.c_double * 3),
                ("period", C.c_double), ("samples_per_period", C.c_int), ("warmup_periods", C.c_int),
                ("output_periods", C.c_int), ("pad_", C.c_int)]


class fp_tol(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("max_steps", C.c_int),
                ("newton_max_iter", C.c_int), ("refactor_every", C.c_int), ("checkpoint_every", C.c_int),
                ("stages", C.c_int), ("pad_", C.c_int)]


class fp_instance(C.Structure):
    _fields_ = [("h_off", C.c_double * 3), ("theta", C.c_double), ("phi", C.c_double),
                ("K", C.c_double), ("d", C.c_double), ("L", C.c_int), ("flags", C.c_int)]


SUR_LAYERS = 5


class fp_surrogate(C.Structure):
    _fields_ = [("W", C.c_void_p * SUR_LAYERS), ("b", C.c_void_p * SUR_LAYERS), ("in_shift", C.c_void_p),
                ("in_scale", C.c_void_p), ("out_shift", C.c_void_p), ("out_scale", C.c_void_p)]


class fp_surrogate_train(C.Structure):
    _fields_ = [("net", fp_surrogate), ("WT", C.c_void_p * SUR_LAYERS), ("Wm", C.c_void_p * SUR_LAYERS),
                ("bm", C.c_void_p * SUR_LAYERS), ("mW", C.c_void_p * SUR_LAYERS), ("vW", C.c_void_p * SUR_LAYERS),
                ("mb", C.c_void_p * SUR_LAYERS), ("vb", C.c_void_p * SUR_LAYERS)]


assert C.sizeof(fp_instance) == 64
assert C.sizeof(fp_drive) == 96

_lib = None


def lib():
    """Load libfp.so once; raise if it is missing (build it with build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfp.so not built: run `python paper_2106_08040_gb300/build.py` "
                           "(or __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    L.fp_max_degree.restype = i
    L.fp_setup.argtypes = [C.POINTER(fp_material), C.POINTER(fp_drive), C.POINTER(fp_tol), i, C.POINTER(vp)]
    L.fp_setup.restype = i
    L.fp_destroy.argtypes = [vp]
    L.fp_destroy.restype = i
    L.fp_num_samples.argtypes = [vp]
    L.fp_num_samples.restype = i
    L.fp_solve_batch.argtypes = [vp, vp, i, vp, vp, vp, vp, vp]
    L.fp_solve_batch.restype = i
    L.fp_signal.argtypes = [vp, vp, i, i, C.POINTER(d), i, vp, vp]
    L.fp_signal.restype = i
    L.fp_operator_dense.argtypes = [C.POINTER(fp_material), C.POINTER(fp_instance), C.POINTER(d), C.POINTER(d)]
    L.fp_operator_dense.restype = i
    L.fp_grad_workspace_bytes.argtypes = [vp, i]
    L.fp_grad_workspace_bytes.restype = C.c_longlong
    L.fp_grad.argtypes = [vp, vp, i, i, C.POINTER(d), i, vp, vp, vp, vp, vp, C.c_ulonglong, vp]
    L.fp_grad.restype = i
    L.fp_grad_noalloc.argtypes = [vp, vp, i, i, C.POINTER(d), i, vp, vp, vp, vp, vp]
    L.fp_grad_noalloc.restype = i
    f = C.c_float
    L.fp_surrogate_workspace_bytes.argtypes = [i, i]
    L.fp_surrogate_workspace_bytes.restype = C.c_longlong
    L.fp_surrogate_infer.argtypes = [C.POINTER(fp_surrogate), vp, i, vp, vp, C.c_ulonglong, vp, vp]
    L.fp_surrogate_infer.restype = i
    L.fp_surrogate_grad.argtypes = [C.POINTER(fp_surrogate_train), vp, vp, i, vp, C.POINTER(vp), C.POINTER(vp), vp,
                                    C.c_ulonglong, vp, vp]
    L.fp_surrogate_grad.restype = i
    L.fp_surrogate_adam.argtypes = [C.POINTER(fp_surrogate_train), C.POINTER(vp), C.POINTER(vp), f, f, f, f, i, vp]
    L.fp_surrogate_adam.restype = i
    L.fp_sweep_plan.argtypes = [vp, vp, i, i, C.POINTER(vp)]
    L.fp_sweep_plan.restype = i
    L.fp_sweep_order.argtypes = [C.POINTER(fp_material), C.POINTER(fp_drive), i, vp, i, i, C.POINTER(i), C.POINTER(i),
                                 C.POINTER(i), C.POINTER(i)]
    L.fp_sweep_order.restype = i
    L.fp_sweep_run.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.fp_sweep_run.restype = i
    L.fp_sweep_autotune.argtypes = [vp, vp, vp, vp, vp, i, vp]
    L.fp_sweep_autotune.restype = i
    L.fp_sweep_info.argtypes = [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i),
                                C.POINTER(f)]
    L.fp_sweep_info.restype = i
    L.fp_sweep_destroy.argtypes = [vp]
    L.fp_sweep_destroy.restype = i
    L.fp_equilibrium.argtypes = [vp, vp, i, vp, vp, vp]
    L.fp_equilibrium.restype = i
    L.fp_m1_fit.argtypes = [vp, i, vp, i, i, i, vp, vp, vp, vp]
    L.fp_m1_fit.restype = i
    L.fp_nrmse.argtypes = [vp, i, i, i, vp, i, vp, vp, vp]
    L.fp_nrmse.restype = i
    L.fp_mixing_order.argtypes = [i, i, C.POINTER(i), C.POINTER(i)]
    L.fp_mixing_order.restype = i
    L.fp_freq_index_set.argtypes = [i, i, i, i, C.POINTER(i), i, C.POINTER(i)]
    L.fp_freq_index_set.restype = i
    L.fp_truncation_degree.argtypes = [C.POINTER(fp_material), C.POINTER(fp_drive), vp, i, i, i, C.POINTER(i)]
    L.fp_truncation_degree.restype = i
    L.fp_m2_gram_bytes.argtypes = [i]
    L.fp_m2_gram_bytes.restype = C.c_longlong
    L.fp_m2_gram.argtypes = [vp, vp, vp, vp, i, i, i, i, i, vp, i, vp, vp]
    L.fp_m2_gram.restype = i
    L.fp_m2_solve.argtypes = [C.POINTER(d), i, i, C.POINTER(d), C.POINTER(d), C.POINTER(d), C.POINTER(d)]
    L.fp_m2_solve.restype = i
    L.fp_surrogate_infer_ensemble.argtypes = [C.POINTER(fp_surrogate), C.POINTER(fp_surrogate), vp, i, vp, vp, vp,
                                              C.c_ulonglong, vp, vp]
    L.fp_surrogate_infer_ensemble.restype = i
    L.fp_peak_fp64.argtypes = [C.POINTER(d)]
    L.fp_peak_fp64.restype = i
    L.fp_status_str.argtypes = [i]
    L.fp_status_str.restype = C.c_char_p
    L.fp_last_error.restype = C.c_char_p
    _lib = L
    return L


def check(rc, what):
    if rc != FP_OK:
        msg = lib().fp_last_error().decode(errors="replace")
        raise RuntimeError("%s failed (%d): %s" % (what, rc, msg))
    return rc

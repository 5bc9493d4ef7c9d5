"""ctypes binding of libsg (C ABI declared in include/sg.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Device blocks are torch CUDA tensors of shape [P, ld] (mode-major,
row a = PCE mode a, contiguous), passed by data pointer with the current
torch stream.  If libsg.so is missing the calls raise; there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsg.so")

SG_OK, SG_NOT_CONVERGED = 0, 1
STATUS_NAMES = {0: "SG_OK", 1: "SG_NOT_CONVERGED", -1: "SG_ERR_ARG", -2: "SG_ERR_CUDA",
                -3: "SG_ERR_NOMEM", -4: "SG_ERR_BREAKDOWN", -5: "SG_ERR_TIMEOUT",
                -6: "SG_ERR_UNSUPPORTED"}
SG_F64, SG_F32 = 0, 1


class SgError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__("%s -> %s: %s" % (fn, STATUS_NAMES.get(status, status), msg))
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int)]


class KlDesc(ctypes.Structure):
    _fields_ = [("sigma2", ctypes.c_double), ("bx", ctypes.c_double), ("by", ctypes.c_double),
                ("g0", ctypes.c_double), ("L", ctypes.c_int),
                ("user_modes", ctypes.POINTER(ctypes.c_double))]


class PrecondOpts(ctypes.Structure):
    _fields_ = [("sx", ctypes.c_int), ("sy", ctypes.c_int), ("overlap", ctypes.c_int),
                ("omega", ctypes.c_double), ("inner_rtol", ctypes.c_double),
                ("inner_max", ctypes.c_int), ("smoother", ctypes.c_int), ("host_loops", ctypes.c_int),
                ("ras_modes", ctypes.c_int), ("inner_orth_passes", ctypes.c_int),
                ("amg_kernel", ctypes.c_int), ("ras_stages", ctypes.c_int),
                ("ras_kernel", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_it", ctypes.c_int), ("restart", ctypes.c_int),
                ("mode", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("max_ir", ctypes.c_int),
                ("hist_host", ctypes.POINTER(ctypes.c_double)), ("hist_cap", ctypes.c_int),
                ("no_fallback", ctypes.c_int), ("orth_passes", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("outer_it", ctypes.c_int), ("inner_it", ctypes.c_int), ("ir_steps", ctypes.c_int),
                ("fallback_used", ctypes.c_int), ("hist_len", ctypes.c_int),
                ("relres", ctypes.c_double), ("t_setup", ctypes.c_double), ("t_solve", ctypes.c_double)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int), ("epochs", ctypes.c_int), ("batch", ctypes.c_int),
                ("lr", ctypes.c_float), ("seed", ctypes.c_uint64), ("target_rtol", ctypes.c_double),
                ("keep_weights", ctypes.c_int), ("loss", ctypes.c_int)]


class TrainInfo(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int), ("steps", ctypes.c_int), ("harvest_solves", ctypes.c_int),
                ("target_its", ctypes.c_int), ("target_relres", ctypes.c_double),
                ("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double),
                ("omega_cnn", ctypes.c_double), ("t_harvest", ctypes.c_double),
                ("t_targets", ctypes.c_double), ("t_train", ctypes.c_double)]


_lib = None
vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
P_i32, P_i64, P_f64 = ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(f64)

# name -> argtypes (restype is always int = sg_status, except sg_last_error)
SIGNATURES = {
    "sg_setup": [ctypes.POINTER(MeshDesc), ctypes.POINTER(KlDesc), ctypes.c_int, ctypes.c_int,
                 ctypes.POINTER(vp)],
    "sg_destroy": [vp],
    "sg_get_sizes": [vp, P_i64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), P_i64, P_i64],
    "sg_get_multi_indices": [vp, P_i32, ctypes.c_int],
    "sg_get_triples": [vp, P_i32, P_i64, P_f64],
    "sg_get_csr": [vp, P_i32, P_i32],
    "sg_get_values": [vp, P_f64],
    "sg_get_rhs": [vp, vp, i64, vp],
    "sg_apply": [vp, ctypes.c_int, vp, i64, vp, i64, vp],
    "sg_residual": [vp, ctypes.c_int, vp, i64, vp, i64, vp, i64, vp],
    "sg_precond_setup": [vp, ctypes.POINTER(PrecondOpts), vp],
    "sg_precond_info": [vp, P_f64, ctypes.POINTER(ctypes.c_int), P_i64, ctypes.POINTER(ctypes.c_int)],
    "sg_get_partition": [vp, ctypes.c_int, P_i32, P_i64, P_i32],
    "sg_precond_stats": [vp, P_f64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(ctypes.c_int)],
    "sg_get_coarse_csr": [vp, P_i64, P_i64, P_i32, P_i32],
    "sg_get_amg_level": [vp, ctypes.c_int, P_i64, P_i32],
    "sg_precond_apply": [vp, ctypes.c_int, ctypes.c_int, vp, i64, vp, i64, vp],
    "sg_solve": [vp, vp, i64, vp, i64, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp],
    "sg_profile": [vp, ctypes.c_int],
    "sg_mdot": [vp, ctypes.c_int, vp, i64, ctypes.c_int, vp, i64, vp, vp],
    "sg_mdot_noalloc": [ctypes.c_int, vp, i64, ctypes.c_int, vp, i64, vp, vp],
    "sg_set_apply_kernel": [vp, ctypes.c_int],
    "sg_set_apply_fp64": [vp, ctypes.c_int],
    "sg_precond_save": [vp, vp, P_i64],
    "sg_set_wait_limit": [vp, ctypes.c_int],
    "sg_newton": [vp, vp, ctypes.c_int64, ctypes.c_double, ctypes.c_int, vp, vp, vp],
    "sg_nonlinear_residual": [vp, vp, i64, vp, i64, vp, i64, vp],
    "sg_sample_solve": [vp, vp, i64, ctypes.c_int, vp, i64, ctypes.c_double, ctypes.c_int,
                        ctypes.POINTER(ctypes.c_int), vp],
    "sg_nonlinear_jacobian_apply": [vp, ctypes.c_int, vp, i64, vp, i64, vp, i64, vp],
    "sg_fourfold_products": [ctypes.c_int, ctypes.c_int, ctypes.c_int, P_i64, P_i32, P_i64, P_f64],
    "sg_precond_load": [vp, vp, ctypes.c_int64],
    "sg_apply_fp64_info": [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), P_i64],
    "sg_set_refine_residual": [vp, ctypes.c_int],
    "sg_refine_residual_info": [vp, ctypes.POINTER(ctypes.c_int), P_i64],
    "sg_residual_refine": [vp, vp, i64, vp, i64, vp, i64, vp],
    "sg_apply_config": [vp] + [ctypes.c_int] * 10,
    "sg_apply_autotune": [vp, ctypes.c_int, ctypes.c_int, P_f64],
    "sg_apply_flux": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "sg_apply_info": [vp, ctypes.c_int, P_i32, P_f64],
    "sg_launch_count": [P_i64],
    "sg_profile_read": [vp, ctypes.c_int, P_i64, P_f64],
    "sg_cnn_init": [vp, ctypes.c_uint64, vp],
    "sg_cnn_set_weights": [vp, ctypes.POINTER(ctypes.c_float), i64, vp],
    "sg_cnn_get_weights": [vp, ctypes.POINTER(ctypes.c_float), i64, ctypes.c_int, vp],
    "sg_cnn_apply": [vp, vp, i64, vp, i64, ctypes.c_int, vp],
    "sg_cnn_train_step": [vp, vp, i64, vp, i64, ctypes.c_int, ctypes.c_float, ctypes.c_int, P_f64, vp],
    "sg_mean_solve": [vp, vp, i64, vp, i64, ctypes.c_int, f64, ctypes.c_int, P_f64,
                      ctypes.POINTER(ctypes.c_int), vp],
    "sg_train_precond": [vp, ctypes.POINTER(TrainOpts), ctypes.POINTER(TrainInfo), vp],
    "sg_cnn_set_loss": [vp, ctypes.c_int],
    "sg_cnn_set_kernel": [vp, ctypes.c_int],
    "sg_precond_set_smoother": [vp, ctypes.c_int, f64, vp],
    "sg_batch_create": [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(SolveOpts), ctypes.POINTER(vp)],
    "sg_batch_solve": [vp, ctypes.POINTER(vp), P_i64, ctypes.POINTER(vp), P_i64, ctypes.POINTER(SolveInfo), vp],
    "sg_batch_destroy": [vp],
    "sg_solve_batch": [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), P_i64, ctypes.POINTER(vp), P_i64,
                       ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo), vp],
}

# functions whose result is not an sg_status: name -> (argtypes, restype)
VALUE_FUNCTIONS = {
    "sg_cnn_param_count": ([], ctypes.c_int64),
}


def lib():
    """Load libsg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsg.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        for name, (args, res) in VALUE_FUNCTIONS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        L.sg_last_error.argtypes = []
        L.sg_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def check(fn, status, allow=(SG_OK,)):
    if status not in allow:
        raise SgError(fn, status, lib().sg_last_error().decode(errors="replace"))
    return status


def call(name, *args, allow=(SG_OK,)):
    return check(name, getattr(lib(), name)(*args), allow)


def ptr(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def stream_handle(stream=None):
    """cudaStream_t of a torch stream (current stream by default)."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def dev_ptr(t):
    return ctypes.c_void_p(t.data_ptr())

"""GB300 (sm_103a) stochastic Galerkin solver of arXiv 2310.14649.

Python face of the C ABI in include/sg.h.  Function names follow the C
entry points; each call only marshals arguments and checks the status code.
Device blocks are torch CUDA tensors [P, ld] (mode-major).
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import SG_F32, SG_F64, SgError, call, dev_ptr, stream_handle

__all__ = ["Problem", "sg_setup", "sg_destroy", "sg_get_sizes", "sg_get_multi_indices",
           "sg_get_triples", "sg_get_csr", "sg_get_values", "sg_get_rhs", "sg_apply",
           "sg_residual", "sg_precond_setup", "sg_precond_info", "sg_get_partition",
           "sg_get_coarse_csr", "sg_get_amg_level", "sg_precond_apply", "sg_solve",
           "sg_profile", "sg_profile_read", "sg_launch_count", "sg_set_apply_kernel", "sg_set_apply_fp64",
           "sg_apply_fp64_info", "sg_set_refine_residual", "sg_refine_residual_info", "sg_residual_refine", "sg_precond_save", "sg_precond_load", "sg_fourfold_products",
           "sg_newton", "sg_nonlinear_residual", "sg_nonlinear_jacobian_apply", "sg_sample_solve",
           "sg_set_wait_limit", "sg_apply_flux",
           "sg_apply_config", "sg_apply_autotune", "sg_apply_info", "sg_mdot",
           "sg_mdot_noalloc", "sg_precond_stats", "sg_precond_ras_kernel", "sg_cnn_param_count", "sg_cnn_init", "sg_cnn_set_weights",
           "sg_cnn_get_weights", "sg_cnn_apply", "sg_cnn_train_step", "sg_mean_solve",
           "sg_train_precond", "sg_precond_set_smoother", "cnn_flatten", "cnn_unflatten", "sg_cnn_set_loss", "sg_cnn_set_kernel",
           "Batch", "sg_batch_create", "sg_batch_solve", "sg_batch_destroy", "sg_solve_batch",
           "SgError", "SG_F32", "SG_F64", "PC_TWOLEVEL", "PC_SMOOTH", "PC_COARSE", "PC_AMG",
           "PC_COARSE_APPLY", "PC_RESTRICT", "PC_INTERP", "PC_RAS_LOCAL", "PC_LEARNED",
           "PC_NETWORK"]

# operators of sg_precond_apply
(PC_TWOLEVEL, PC_SMOOTH, PC_COARSE, PC_AMG, PC_COARSE_APPLY, PC_RESTRICT, PC_INTERP,
 PC_RAS_LOCAL, PC_LEARNED, PC_NETWORK) = range(10)

# channels of the learned smoother's convolution layers
CNN_CHANNELS = (2, 32, 32, 32, 32, 1)


class Problem:
    """Owning wrapper of an sg_problem handle."""

    def __init__(self, handle, L):
        self.handle = handle
        self.L = L
        n, P, K, nnz, T = sg_get_sizes(self)
        self.n, self.P, self.K, self.nnzA, self.T = n, P, K, nnz, T

    def close(self):
        if self.handle:
            sg_destroy(self)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sg_setup(N, L, p_out, q_in, sigma2=0.3, bx=0.5, by=0.5, g0=0.0, user_modes=None):
    mesh = _lib.MeshDesc(N)
    um = None
    if user_modes is not None:
        um = np.ascontiguousarray(user_modes, dtype=np.float64)
    kl = _lib.KlDesc(sigma2, bx, by, g0, L,
                     um.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if um is not None else None)
    h = ctypes.c_void_p()
    call("sg_setup", ctypes.byref(mesh), ctypes.byref(kl), p_out, q_in, ctypes.byref(h))
    return Problem(h, L)


def sg_destroy(prob):
    call("sg_destroy", prob.handle)


def sg_get_sizes(prob):
    n, nnz, T = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    P, K = ctypes.c_int(), ctypes.c_int()
    call("sg_get_sizes", prob.handle, ctypes.byref(n), ctypes.byref(P), ctypes.byref(K),
         ctypes.byref(nnz), ctypes.byref(T))
    return n.value, P.value, K.value, nnz.value, T.value


def sg_get_multi_indices(prob, which):
    rows = prob.P if which == 0 else prob.K
    L = prob.L
    out = np.zeros((rows, max(L, 0)), dtype=np.int32)
    if L > 0:
        call("sg_get_multi_indices", prob.handle, _lib.ptr(out, ctypes.c_int32), which)
    return out


def sg_get_triples(prob):
    kab = np.zeros((prob.T, 3), dtype=np.int32)
    num = np.zeros(prob.T, dtype=np.int64)
    g = np.zeros(prob.T, dtype=np.float64)
    call("sg_get_triples", prob.handle, _lib.ptr(kab, ctypes.c_int32), _lib.ptr(num, ctypes.c_int64),
         _lib.ptr(g, ctypes.c_double))
    return kab, num, g


def sg_get_csr(prob):
    rowptr = np.zeros(prob.n + 1, dtype=np.int32)
    colidx = np.zeros(prob.nnzA, dtype=np.int32)
    call("sg_get_csr", prob.handle, _lib.ptr(rowptr, ctypes.c_int32), _lib.ptr(colidx, ctypes.c_int32))
    return rowptr, colidx


def sg_get_values(prob):
    vals = np.zeros((prob.K, prob.nnzA), dtype=np.float64)
    call("sg_get_values", prob.handle, _lib.ptr(vals, ctypes.c_double))
    return vals


def sg_get_rhs(prob, F, stream=None):
    call("sg_get_rhs", prob.handle, dev_ptr(F), F.stride(0), stream_handle(stream))


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return SG_F64
    if t.dtype == torch.float32:
        return SG_F32
    raise TypeError("blocks must be float32 or float64 CUDA tensors")


def _check_block(prob, t, name):
    if not t.is_cuda or t.dim() != 2 or t.shape[0] != prob.P or t.stride(1) != 1 or t.shape[1] < prob.n:
        raise ValueError("%s must be a CUDA tensor [P, ld >= n] with unit column stride" % name)


def sg_apply(prob, X, Y, stream=None):
    """Y = sum_k A_k X G_k^T (X, Y: [P, ld] CUDA tensors, same dtype)."""
    _check_block(prob, X, "X")
    _check_block(prob, Y, "Y")
    call("sg_apply", prob.handle, _dtype_code(X), dev_ptr(X), X.stride(0), dev_ptr(Y), Y.stride(0),
         stream_handle(stream))


def sg_residual(prob, F, X, R, stream=None):
    """R = F - sum_k A_k X G_k^T."""
    for t, nm in ((F, "F"), (X, "X"), (R, "R")):
        _check_block(prob, t, nm)
    call("sg_residual", prob.handle, _dtype_code(X), dev_ptr(F), F.stride(0), dev_ptr(X), X.stride(0),
         dev_ptr(R), R.stride(0), stream_handle(stream))


def sg_precond_setup(prob, sx, sy, overlap, omega=0.0, inner_rtol=0.0, inner_max=0, smoother=0,
                     host_loops=False, ras_modes=0, inner_orth_passes=0, amg_kernel=0, ras_stages=0, ras_kernel=0,
                     stream=None):
    opts = _lib.PrecondOpts(sx, sy, overlap, omega, inner_rtol, inner_max, smoother, 1 if host_loops else 0,
                            ras_modes, inner_orth_passes, amg_kernel, ras_stages, ras_kernel)
    call("sg_precond_setup", prob.handle, ctypes.byref(opts), stream_handle(stream))
    prob.nc = sg_precond_info(prob)[2]


def sg_precond_info(prob):
    om, lev, nc, inner = ctypes.c_double(), ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
    call("sg_precond_info", prob.handle, ctypes.byref(om), ctypes.byref(lev), ctypes.byref(nc),
         ctypes.byref(inner))
    return om.value, lev.value, nc.value, inner.value


def sg_precond_stats(prob):
    """(RAS useful flops per application, boxes, padded line width)."""
    f, nb, w = ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    call("sg_precond_stats", prob.handle, ctypes.byref(f), ctypes.byref(nb), ctypes.byref(w), None)
    return f.value, nb.value, w.value


def sg_precond_ras_kernel(prob):
    """The FP32 RAS local-solve kernel in use: 0 line FMA, 1 line TF32 MMA,
    2 explicit local inverses on tcgen05."""
    k = ctypes.c_int()
    call("sg_precond_stats", prob.handle, None, None, None, ctypes.byref(k))
    return k.value


def sg_get_partition(prob, sub):
    cnt = ctypes.c_int64()
    call("sg_get_partition", prob.handle, sub, None, ctypes.byref(cnt), None)
    idx = np.zeros(cnt.value, dtype=np.int32)
    own = np.zeros(cnt.value, dtype=np.int32)
    call("sg_get_partition", prob.handle, sub, _lib.ptr(idx, ctypes.c_int32), ctypes.byref(cnt),
         _lib.ptr(own, ctypes.c_int32))
    return idx, own


def sg_get_coarse_csr(prob):
    nc, nnz = ctypes.c_int64(), ctypes.c_int64()
    call("sg_get_coarse_csr", prob.handle, ctypes.byref(nc), ctypes.byref(nnz), None, None)
    rp = np.zeros(nc.value + 1, dtype=np.int32)
    ci = np.zeros(nnz.value, dtype=np.int32)
    call("sg_get_coarse_csr", prob.handle, None, None, _lib.ptr(rp, ctypes.c_int32), _lib.ptr(ci, ctypes.c_int32))
    return rp, ci


def sg_get_amg_level(prob, level):
    n = ctypes.c_int64()
    call("sg_get_amg_level", prob.handle, level, ctypes.byref(n), None)
    agg = np.full(n.value, -1, dtype=np.int32)
    call("sg_get_amg_level", prob.handle, level, ctypes.byref(n), _lib.ptr(agg, ctypes.c_int32))
    return n.value, agg


def sg_precond_apply(prob, which, R, Z, stream=None):
    """Z = op(R) for one piece of the two-level preconditioner (PC_*)."""
    if not (R.is_cuda and Z.is_cuda and R.dtype == Z.dtype and R.stride(1) == 1 and Z.stride(1) == 1):
        raise ValueError("R and Z must be CUDA tensors [P, ld] of one dtype")
    call("sg_precond_apply", prob.handle, _dtype_code(R), which, dev_ptr(R), R.stride(0), dev_ptr(Z),
         Z.stride(0), stream_handle(stream))


def sg_solve(prob, X, F=None, rtol=1e-8, max_it=500, restart=30, mode=0, inner_rtol=0.0, max_ir=0,
             hist_cap=256, stream=None, allow_not_converged=False, fallback=True, orth_passes=0):
    """Solve sum_k A_k X G_k^T = F (F None: the load vector).  X (FP64, [P, ld])
    holds the initial guess and receives the solution.  Returns a dict of
    the solve info (and the residual history)."""
    import torch
    _check_block(prob, X, "X")
    if X.dtype != torch.float64 or (F is not None and F.dtype != torch.float64):
        raise TypeError("sg_solve works on FP64 blocks")
    hist = np.zeros(max(hist_cap, 1), dtype=np.float64)
    opts = _lib.SolveOpts(rtol, max_it, restart, mode, inner_rtol, max_ir,
                          hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), hist_cap,
                          0 if fallback else 1, orth_passes)
    info = _lib.SolveInfo()
    allow = (0, 1) if allow_not_converged else (0,)
    st = call("sg_solve", prob.handle, dev_ptr(F) if F is not None else None,
              F.stride(0) if F is not None else 0, dev_ptr(X), X.stride(0), ctypes.byref(opts),
              ctypes.byref(info), stream_handle(stream), allow=allow)
    out = {f: getattr(info, f) for f, _ in _lib.SolveInfo._fields_}
    out["hist"] = hist[:info.hist_len].copy()
    out["status"] = st
    return out


def sg_newton(prob, X, tol_update=1e-8, max_newton=20, max_it=500, restart=30, mode=1, inner_rtol=0.0,
              hist_cap=64, stream=None, allow_not_converged=False, orth_passes=0):
    """Newton's method for -div(c (1 + u^2) grad u) = 1 from the initial
    guess in X (FP64, [P, ld]; the solution on return).  Returns a dict of
    the solve info (ir_steps = Newton steps, hist = relative updates)."""
    import torch
    _check_block(prob, X, "X")
    if X.dtype != torch.float64:
        raise TypeError("sg_newton works on FP64 blocks")
    hist = np.zeros(max(hist_cap, 1), dtype=np.float64)
    opts = _lib.SolveOpts(1e-8, max_it, restart, mode, inner_rtol, 0,
                          hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), hist_cap, 0, orth_passes)
    info = _lib.SolveInfo()
    allow = (0, 1) if allow_not_converged else (0,)
    st = call("sg_newton", prob.handle, dev_ptr(X), X.stride(0), ctypes.c_double(tol_update), max_newton,
              ctypes.byref(opts), ctypes.byref(info), stream_handle(stream), allow=allow)
    out = {f: getattr(info, f) for f, _ in _lib.SolveInfo._fields_}
    out["hist"] = hist[:info.hist_len].copy()
    out["status"] = st
    return out


def sg_nonlinear_residual(prob, X, R, F=None, stream=None):
    """R = F - A(X) X of the nonlinear problem (FP64 blocks; F None: the
    load vector)."""
    _check_block(prob, X, "X")
    _check_block(prob, R, "R")
    call("sg_nonlinear_residual", prob.handle, dev_ptr(F) if F is not None else None,
         F.stride(0) if F is not None else 0, dev_ptr(X), X.stride(0), dev_ptr(R), R.stride(0),
         stream_handle(stream))


def sg_nonlinear_jacobian_apply(prob, U, dU, Y, stream=None):
    """Y = J(U) dU of the nonlinear problem (FP32 or FP64 blocks of one
    dtype)."""
    for t, nm in ((U, "U"), (dU, "dU"), (Y, "Y")):
        _check_block(prob, t, nm)
    if not (U.dtype == dU.dtype == Y.dtype):
        raise TypeError("U, dU and Y must have one dtype")
    call("sg_nonlinear_jacobian_apply", prob.handle, _dtype_code(U), dev_ptr(U), U.stride(0), dev_ptr(dU),
         dU.stride(0), dev_ptr(Y), Y.stride(0), stream_handle(stream))


def sg_sample_solve(prob, xi, U, rtol=1e-6, max_it=2000, stream=None, allow_not_converged=False):
    """Deterministic solves for Monte Carlo samples: xi (CUDA float64
    [S, L]) -> U (CUDA float32 or float64 [S, ld >= n], row s = u_s).
    Returns the largest CG iteration count."""
    import torch
    if xi.dtype != torch.float64 or not xi.is_contiguous() or xi.dim() != 2 or xi.shape[1] != prob.L:
        raise TypeError("xi must be a contiguous float64 [S, L] tensor")
    if U.dim() != 2 or U.shape[0] != xi.shape[0] or U.shape[1] < prob.n or U.stride(1) != 1:
        raise ValueError("U must be [S, ld >= n] with unit column stride")
    its = ctypes.c_int(0)
    allow = (0, 1) if allow_not_converged else (0,)
    call("sg_sample_solve", prob.handle, dev_ptr(xi), xi.shape[0], _dtype_code(U), dev_ptr(U), U.stride(0),
         ctypes.c_double(rtol), max_it, ctypes.byref(its), stream_handle(stream), allow=allow)
    return its.value


def sg_profile(prob, enable):
    call("sg_profile", prob.handle, 1 if enable else 0)


def sg_profile_read(prob, kind):
    """(launches, total ms) of one kind: kernels 0 fine apply FP32, 1 fine
    apply FP64, 2 coarse apply FP32, 3 coarse apply FP64, 4/5 RAS local
    solve FP32/FP64; phases 6 smoother, 7 coarse correction, 8 Arnoldi
    step, 9 refinement bookkeeping."""
    cnt, ms = ctypes.c_int64(), ctypes.c_double()
    call("sg_profile_read", prob.handle, kind, ctypes.byref(cnt), ctypes.byref(ms))
    return cnt.value, ms.value


def sg_launch_count():
    c = ctypes.c_int64()
    call("sg_launch_count", ctypes.byref(c))
    return c.value


def sg_set_apply_kernel(prob, mode):
    """0 auto, 1 shared-memory kernel, 2 register-specialised kernel."""
    call("sg_set_apply_kernel", prob.handle, mode)


def sg_set_apply_fp64(prob, mode):
    """FP64 applies over assembled P x P edge blocks: 0 auto (memory
    permitting), 1 never, 2 always."""
    call("sg_set_apply_fp64", prob.handle, mode)


def sg_precond_save(prob):
    """The learned smoother (weights, damping, selection) as bytes."""
    n = ctypes.c_int64()
    call("sg_precond_save", prob.handle, None, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value)
    call("sg_precond_save", prob.handle, buf, ctypes.byref(n))
    return buf.raw[:n.value]


def sg_precond_load(prob, data):
    """Restores what sg_precond_save returned."""
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    call("sg_precond_load", prob.handle, buf, len(data))


def sg_fourfold_products(L, p, q):
    """Nonzero <psi_i psi_j psi_k psi_l> (host-only): (ijkl int32 [T4, 4],
    num int64 [T4], t float64 [T4])."""
    n = ctypes.c_int64(0)
    call("sg_fourfold_products", L, p, q, ctypes.byref(n), None, None, None)
    ijkl = np.zeros((n.value, 4), dtype=np.int32)
    num = np.zeros(n.value, dtype=np.int64)
    t = np.zeros(n.value, dtype=np.float64)
    call("sg_fourfold_products", L, p, q, ctypes.byref(n), _lib.ptr(ijkl, ctypes.c_int32),
         _lib.ptr(num, ctypes.c_int64), _lib.ptr(t, ctypes.c_double))
    return ijkl, num, t


def sg_set_refine_residual(prob, mode):
    """Refinement residuals: 0 auto (double-FP32 edge blocks, memory
    permitting), 1 FP64 apply, 2 always double-FP32."""
    call("sg_set_refine_residual", prob.handle, mode)


def sg_refine_residual_info(prob):
    b, nb = ctypes.c_int(), ctypes.c_int64()
    call("sg_refine_residual_info", prob.handle, ctypes.byref(b), ctypes.byref(nb))
    return {"built": b.value, "bytes": nb.value}


def sg_residual_refine(prob, F, X, R, stream=None):
    """R = F - sum_k A_k X G_k^T as the refinement forms it (FP64 blocks)."""
    for t, nm in ((F, "F"), (X, "X"), (R, "R")):
        _check_block(prob, t, nm)
    if any(_dtype_code(t) != SG_F64 for t in (F, X, R)):
        raise TypeError("sg_residual_refine: FP64 blocks only")
    call("sg_residual_refine", prob.handle, dev_ptr(F), F.stride(0), dev_ptr(X), X.stride(0), dev_ptr(R),
         R.stride(0), stream_handle(stream))


def sg_apply_fp64_info(prob):
    f, c, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    call("sg_apply_fp64_info", prob.handle, ctypes.byref(f), ctypes.byref(c), ctypes.byref(b))
    return {"fine": f.value, "coarse": c.value, "bytes": b.value}


def sg_apply_config(prob, rows=1, groups=1, igroups=1, sgroups=1, prefetch=8, min_blocks=1, stages=0, cgroups=1,
                    warps=4, which=0):
    call("sg_apply_config", prob.handle, which, rows, groups, igroups, sgroups, prefetch, min_blocks, stages, cgroups,
         warps)


def sg_apply_flux(prob, mode=-1):
    """Edge-flux form of the fine FP32 operator: 0 slot form, 1 edge form,
    2 autotuner decides, -1 query.  Returns 1 when the edge form is used."""
    on = ctypes.c_int(0)
    call("sg_apply_flux", prob.handle, mode, ctypes.byref(on))
    return on.value


def sg_apply_autotune(prob, force=False, which=0):
    ms = ctypes.c_double()
    call("sg_apply_autotune", prob.handle, which, 1 if force else 0, ctypes.byref(ms))
    return ms.value


def sg_apply_info(prob, which=0):
    cfg = np.zeros(10, dtype=np.int32)
    cs = ctypes.c_double()
    call("sg_apply_info", prob.handle, which, _lib.ptr(cfg, ctypes.c_int32), ctypes.byref(cs))
    keys = ["rows", "groups", "igroups", "sgroups", "prefetch", "min_blocks", "stages", "cgroups", "warps",
            "generator"]
    out = {k: int(v) for k, v in zip(keys, cfg)}
    out["compile_s"] = cs.value
    return out


def sg_mdot(prob, V, w, out, stream=None):
    """out[i] = V[i] . w for the rows of a [nv, len] CUDA tensor V (float32
    or float64) and a vector w of the same dtype; out: float64 CUDA [nv]."""
    if V.dtype != w.dtype or out.dtype.itemsize != 8 or V.stride(1) != 1:
        raise TypeError("V, w of one dtype (row-contiguous V), out float64")
    call("sg_mdot", prob.handle, _dtype_code(V), dev_ptr(V), V.stride(0), V.shape[0], dev_ptr(w), V.shape[1],
         dev_ptr(out), stream_handle(stream))


def sg_mdot_noalloc(V, w, out, stream=None):
    """sg_mdot without a handle and without any device allocation (static
    scratch inside the library); calls that overlap on the GPU race."""
    if V.dtype != w.dtype or out.dtype.itemsize != 8 or V.stride(1) != 1:
        raise TypeError("V, w of one dtype (row-contiguous V), out float64")
    call("sg_mdot_noalloc", _dtype_code(V), dev_ptr(V), V.stride(0), V.shape[0], dev_ptr(w), V.shape[1],
         dev_ptr(out), stream_handle(stream))


# ---------------------------------------------------------------------------
# learned smoother
# ---------------------------------------------------------------------------
def sg_cnn_param_count():
    return int(_lib.lib().sg_cnn_param_count())


def cnn_flatten(params):
    """[(W [3,3,Cin,Cout], b [Cout])] per layer -> the flat FP32 array of the ABI."""
    parts = []
    for W, b in params:
        parts.append(np.asarray(W, dtype=np.float32).ravel())
        parts.append(np.asarray(b, dtype=np.float32).ravel())
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)


def cnn_unflatten(flat):
    """Inverse of cnn_flatten (float64 arrays)."""
    out, off = [], 0
    for l in range(5):
        ci, co = CNN_CHANNELS[l], CNN_CHANNELS[l + 1]
        W = np.asarray(flat[off:off + 9 * ci * co], dtype=np.float64).reshape(3, 3, ci, co)
        off += 9 * ci * co
        b = np.asarray(flat[off:off + co], dtype=np.float64)
        off += co
        out.append((W, b))
    return out


def sg_cnn_init(prob, seed=0, stream=None):
    call("sg_cnn_init", prob.handle, seed, stream_handle(stream))


def sg_cnn_set_weights(prob, params, stream=None):
    """params: flat FP32 array or [(W, b)] per layer."""
    flat = params if isinstance(params, np.ndarray) else cnn_flatten(params)
    flat = np.ascontiguousarray(flat, dtype=np.float32)
    call("sg_cnn_set_weights", prob.handle, _lib.ptr(flat, ctypes.c_float), flat.size, stream_handle(stream))


def sg_cnn_get_weights(prob, gradient=False, stream=None):
    """Flat FP32 weights (or the last step's gradient)."""
    flat = np.zeros(sg_cnn_param_count(), dtype=np.float32)
    call("sg_cnn_get_weights", prob.handle, _lib.ptr(flat, ctypes.c_float), flat.size, 1 if gradient else 0,
         stream_handle(stream))
    return flat


def _check_images(prob, t, name):
    import torch
    if not t.is_cuda or t.dtype != torch.float32 or t.dim() != 2 or t.stride(1) != 1 or t.shape[1] < prob.n:
        raise ValueError("%s must be a float32 CUDA tensor [nimg, ld >= n]" % name)


def sg_cnn_apply(prob, R, Z, stream=None):
    """Z[a] = rms(R[a]) CNN(features(R[a])) for every row a of R (Z rows
    are written up to their stride: Z must be contiguous)."""
    _check_images(prob, R, "R")
    _check_images(prob, Z, "Z")
    if not Z.is_contiguous():
        raise ValueError("Z must be contiguous")
    call("sg_cnn_apply", prob.handle, dev_ptr(R), R.stride(0), dev_ptr(Z), Z.stride(0), R.shape[0],
         stream_handle(stream))


def sg_cnn_train_step(prob, R, Zstar, lr=1e-3, update=True, stream=None):
    """One step on (R[a], Zstar[a]) pairs; returns the loss before the update."""
    _check_images(prob, R, "R")
    _check_images(prob, Zstar, "Zstar")
    loss = ctypes.c_double()
    call("sg_cnn_train_step", prob.handle, dev_ptr(R), R.stride(0), dev_ptr(Zstar), Zstar.stride(0), R.shape[0],
         lr, 1 if update else 0, ctypes.byref(loss), stream_handle(stream))
    return loss.value


def sg_cnn_set_kernel(prob, kind):
    """Forward convolutions: 1 tcgen05 (default), 0 mma.sync."""
    call("sg_cnn_set_kernel", prob.handle, kind)


def sg_set_wait_limit(prob, limit=-1):
    """Polls of a tcgen05 completion wait (network convolutions, RAS
    inverse products) before SG_ERR_TIMEOUT (-1: default; 0: every wait
    runs out at once)."""
    call("sg_set_wait_limit", prob.handle, limit)


def sg_cnn_set_loss(prob, kind):
    """Loss of sg_cnn_train_step: 0 energy norm of A_0, 1 relative L2 error."""
    call("sg_cnn_set_loss", prob.handle, kind)


def sg_mean_solve(prob, B, Z, rtol=1e-6, max_it=500, stream=None):
    """Z[a] = A_0^{-1} B[a] (float32 CUDA rows); returns (worst relres, its)."""
    _check_images(prob, B, "B")
    _check_images(prob, Z, "Z")
    rel, its = ctypes.c_double(), ctypes.c_int()
    call("sg_mean_solve", prob.handle, dev_ptr(B), B.stride(0), dev_ptr(Z), Z.stride(0), B.shape[0], rtol,
         max_it, ctypes.byref(rel), ctypes.byref(its), stream_handle(stream))
    return rel.value, its.value


def sg_train_precond(prob, n_pairs=4096, epochs=12, batch=32, lr=1e-3, seed=0, target_rtol=1e-6,
                     keep_weights=False, loss=0, stream=None):
    """Harvest residuals, build A_0^{-1} targets, train, select the learned
    smoother.  loss: 0 energy norm of A_0, 1 relative L2 error."""
    opts = _lib.TrainOpts(n_pairs, epochs, batch, lr, seed, target_rtol, 1 if keep_weights else 0, loss)
    info = _lib.TrainInfo()
    call("sg_train_precond", prob.handle, ctypes.byref(opts), ctypes.byref(info), stream_handle(stream))
    return {f: getattr(info, f) for f, _ in _lib.TrainInfo._fields_}


def sg_precond_set_smoother(prob, smoother, omega=0.0, stream=None):
    """0 RAS, 1 learned (omega <= 0: estimate)."""
    call("sg_precond_set_smoother", prob.handle, smoother, omega, stream_handle(stream))


# ---------------------------------------------------------------------------
# graph-captured batches of systems
# ---------------------------------------------------------------------------
class Batch:
    """Owning wrapper of an sg_batch handle (keeps its problems alive)."""

    def __init__(self, handle, probs):
        self.handle = handle
        self.probs = list(probs)

    def close(self):
        if self.handle:
            sg_batch_destroy(self)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _solve_opts(rtol, max_it, restart, mode, inner_rtol, max_ir, orth_passes=0):
    return _lib.SolveOpts(rtol, max_it, restart, mode, inner_rtol, max_ir, None, 0, 0, orth_passes)


def _ptr_array(ts, allow_none=False):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if (t is None and allow_none) else t.data_ptr()
    return arr


def _ld_array(ts):
    arr = (ctypes.c_int64 * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = 0 if t is None else t.stride(0)
    return arr


def sg_batch_create(probs, rtol=1e-8, max_it=500, restart=30, mode=1, inner_rtol=0.0, max_ir=0, orth_passes=0):
    handles = (ctypes.c_void_p * len(probs))(*[p.handle.value for p in probs])
    opts = _solve_opts(rtol, max_it, restart, mode, inner_rtol, max_ir, orth_passes)
    h = ctypes.c_void_p()
    call("sg_batch_create", handles, len(probs), ctypes.byref(opts), ctypes.byref(h))
    return Batch(h, probs)


def _infos_out(infos, sts):
    out = []
    for inf in infos:
        d = {f: getattr(inf, f) for f, _ in _lib.SolveInfo._fields_}
        d["status"] = sts
        out.append(d)
    return out


def sg_batch_solve(batch, Xs, Fs=None, stream=None, allow_not_converged=False):
    """Solve all systems of the batch (Xs: FP64 [P_i, ld_i] CUDA tensors,
    guesses in, solutions out; Fs: None or per-system FP64 blocks / None)."""
    import torch
    for p, X in zip(batch.probs, Xs):
        _check_block(p, X, "X")
        if X.dtype != torch.float64:
            raise TypeError("batch solves work on FP64 blocks")
    Fs = Fs if Fs is not None else [None] * len(Xs)
    infos = (_lib.SolveInfo * len(Xs))()
    allow = (0, 1) if allow_not_converged else (0,)
    st = call("sg_batch_solve", batch.handle, _ptr_array(Fs, True), _ld_array(Fs), _ptr_array(Xs), _ld_array(Xs),
              infos, stream_handle(stream), allow=allow)
    return _infos_out(infos, st)


def sg_batch_destroy(batch):
    call("sg_batch_destroy", batch.handle)


def sg_solve_batch(probs, Xs, Fs=None, rtol=1e-8, max_it=500, restart=30, mode=1, inner_rtol=0.0, max_ir=0,
                   stream=None, allow_not_converged=False, orth_passes=0):
    """One-shot batch: record, solve, release."""
    handles = (ctypes.c_void_p * len(probs))(*[p.handle.value for p in probs])
    opts = _solve_opts(rtol, max_it, restart, mode, inner_rtol, max_ir, orth_passes)
    Fs = Fs if Fs is not None else [None] * len(Xs)
    infos = (_lib.SolveInfo * len(Xs))()
    allow = (0, 1) if allow_not_converged else (0,)
    st = call("sg_solve_batch", handles, len(probs), _ptr_array(Fs, True), _ld_array(Fs), _ptr_array(Xs),
              _ld_array(Xs), ctypes.byref(opts), infos, stream_handle(stream), allow=allow)
    return _infos_out(infos, st)

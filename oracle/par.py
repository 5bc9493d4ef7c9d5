"""Multi-core FP64 oracle solve of the Galerkin system (Sec. 2.1, Eq.
Galerkin_L_exp; GMRES of Sec. 3 with the mean-based block preconditioner).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The arithmetic is the same as ``galerkin.solve_gmres``: restarted
right-preconditioned GMRES with modified Gram-Schmidt and Givens rotations
on the flat mode-major vector, preconditioned by I kron A_0^{-1}.  The
operator apply, the preconditioner's substitutions and the vector kernels
run as plain C loops over all host cores (``sgo.c``, built into
``libsgo.so`` beside it); A_0 is factored once by LAPACK's banded Cholesky
(bandwidth N - 1 in the lexicographic node order).
"""
import ctypes
import os
import subprocess
import time

import numpy as np
import scipy.linalg as sla

from . import galerkin

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sgo.c")
LIB = os.path.join(HERE, "libsgo.so")
_lib = None


def build_lib():
    """Compile sgo.c into libsgo.so with gcc and OpenMP (no host-specific
    instructions, no contracted multiply-adds)."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", SRC, "-o", tmp],
                   check=True, capture_output=True, text=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_lib())
        i64, dp, lp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
        L.sgo_threads.restype = ctypes.c_int
        L.sgo_set_threads.argtypes = [ctypes.c_int]
        L.sgo_apply.argtypes = [i64, ctypes.c_int, ctypes.c_int, lp, lp, i64, dp, i64, lp, dp, dp, dp]
        L.sgo_band_solve.argtypes = [i64, i64, dp, ctypes.c_int, dp, dp]
        L.sgo_dot.argtypes = [i64, dp, dp]
        L.sgo_dot.restype = ctypes.c_double
        L.sgo_axpy.argtypes = [i64, ctypes.c_double, dp, dp]
        L.sgo_scal.argtypes = [i64, ctypes.c_double, dp, dp]
        _lib = L
    return _lib


def threads():
    return lib().sgo_threads()


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _l(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class Operator:
    """The Galerkin operator and its preconditioner on flat mode-major
    vectors, with the arrays laid out once for the C loops."""

    def __init__(self, prob):
        self.prob = prob
        self.n, self.P, self.K = prob.n, prob.P, prob.K
        if self.P > 512:
            raise ValueError("sgo_apply handles at most 512 modes")
        self.rowptr = np.ascontiguousarray(prob.rowptr, dtype=np.int64)
        self.colidx = np.ascontiguousarray(prob.colidx, dtype=np.int64)
        # edge by edge: the K values of one stencil entry side by side
        self.vals_e = np.ascontiguousarray(np.asarray(prob.vals, dtype=np.float64).T)
        self.kab = np.ascontiguousarray(prob.kab, dtype=np.int64)
        self.g = np.ascontiguousarray(prob.g, dtype=np.float64)
        self.nnz = len(self.colidx)
        self.lb = None

    def apply(self, x, y=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x) if y is None else y
        lib().sgo_apply(self.n, self.P, self.K, _l(self.rowptr), _l(self.colidx), self.nnz, _d(self.vals_e),
                        len(self.g), _l(self.kab), _d(self.g), _d(x), _d(y))
        return y

    def factor_mean(self):
        """Banded Cholesky of A_0 (LAPACK), kept by columns for the C
        substitutions."""
        A0 = self.prob.A(0).tocsr()
        bw = self.prob.N - 1
        n = self.n
        ab = np.zeros((bw + 1, n))
        coo = A0.tocoo()
        low = coo.row >= coo.col
        ab[coo.row[low] - coo.col[low], coo.col[low]] = coo.data[low]
        cb = sla.cholesky_banded(ab, lower=True)
        self.bw = bw
        self.lb = np.ascontiguousarray(cb.T)
        return self

    def precond(self, v, out=None):
        if self.lb is None:
            self.factor_mean()
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty_like(v) if out is None else out
        lib().sgo_band_solve(self.n, self.bw, _d(self.lb), self.P, _d(v), _d(out))
        return out


def gmres(op, f, tol=1e-12, restart=50, max_it=2000, x0=None):
    """Restarted right-preconditioned GMRES (modified Gram-Schmidt, Givens
    rotations), the algorithm of ``galerkin.gmres`` with the vector work in
    C.  Stops on the true residual.  Returns (x, iterations, history)."""
    L = lib()
    m = len(f)
    f = np.ascontiguousarray(f, dtype=np.float64)
    nf = np.sqrt(L.sgo_dot(m, _d(f), _d(f)))
    x = np.zeros(m) if x0 is None else np.array(x0, dtype=np.float64)
    hist = []
    its = 0
    if nf == 0.0:
        return x, 0, hist
    V = np.empty((restart + 1, m))
    Z = np.empty((restart, m))
    w = np.empty(m)
    while its < max_it:
        r = f - op.apply(x)
        beta = np.sqrt(L.sgo_dot(m, _d(r), _d(r)))
        if beta / nf <= tol:
            break
        L.sgo_scal(m, 1.0 / beta, _d(r), _d(V[0]))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        gvec = np.zeros(restart + 1)
        gvec[0] = beta
        j_used = 0
        for j in range(restart):
            op.precond(V[j], Z[j])
            op.apply(Z[j], w)
            for i in range(j + 1):
                H[i, j] = L.sgo_dot(m, _d(V[i]), _d(w))
                L.sgo_axpy(m, -H[i, j], _d(V[i]), _d(w))
            H[j + 1, j] = np.sqrt(L.sgo_dot(m, _d(w), _d(w)))
            hnext = H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            its += 1
            j_used = j + 1
            hist.append(abs(gvec[j + 1]) / nf)
            if abs(gvec[j + 1]) / nf <= tol * 0.5 or its >= max_it or hnext == 0.0:
                break
            L.sgo_scal(m, 1.0 / hnext, _d(w), _d(V[j + 1]))
        yv = np.linalg.solve(np.triu(H[:j_used, :j_used]), gvec[:j_used])
        for i in range(j_used):
            L.sgo_axpy(m, yv[i], _d(Z[i]), _d(x))
    return x, its, hist


def solve(prob, F=None, tol=1e-12, restart=50, max_it=2000, op=None, X0=None):
    """GMRES on the Galerkin system, right-preconditioned by I kron A_0^{-1}
    (multi-core).  Returns (X [n, P], iterations, history, seconds of the
    solve excluding the one-time factorisation)."""
    op = op or Operator(prob).factor_mean()
    if op.lb is None:
        op.factor_mean()
    F = prob.rhs() if F is None else F
    x0 = None if X0 is None else galerkin.to_vec(X0)
    t0 = time.perf_counter()
    x, its, hist = gmres(op, galerkin.to_vec(F), tol, restart, max_it, x0)
    dt = time.perf_counter() - t0
    return galerkin.from_vec(x, prob.n, prob.P), its, hist, dt

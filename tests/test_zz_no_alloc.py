"""The allocation-free multi-dot entry point (sg_mdot_noalloc) against the
handle-based sg_mdot and against the host FP64 product, through the C ABI
(GPU).

sg_mdot_noalloc is for callers that cannot call cudaMalloc (a framework's
caching allocator holds the free memory, or the loop cannot afford the
synchronisation an allocation may cause, or there is no handle to own
scratch).  Its scratch is a static device array shared by every call, so
two calls in a row must each give the right answer: the second must not see
the first one's partial sums or counter.  This file is collected last.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U64, U32 = 2.0 ** -53, 2.0 ** -24


def _inputs(nv, length, dtype, seed):
    import torch
    g = torch.Generator().manual_seed(seed)
    V = torch.randn((nv, length + 3), generator=g, dtype=torch.float64).to(dtype).cuda()[:, :length]
    w = torch.randn(length, generator=g, dtype=torch.float64).to(dtype).cuda()
    return V, w


def _noalloc(V, w, out):
    import torch
    from paper_2310_14649_gb300 import _lib
    code = 0 if V.dtype == torch.float64 else 1
    st = _lib.lib().sg_mdot_noalloc(code, ctypes.c_void_p(V.data_ptr()), V.stride(0), V.shape[0],
                                    ctypes.c_void_p(w.data_ptr()), V.shape[1], ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _lib.lib().sg_last_error()


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_matches_mdot_on_two_calls(gpu, dt):
    import torch
    import paper_2310_14649_gb300 as sg
    dtype = torch.float64 if dt == "f64" else torch.float32
    u = U64 if dt == "f64" else U32
    prob = sg.sg_setup(8, 1, 1, 2)
    for seed, (nv, length) in ((1, (32, 250007)), (2, (5, 1031))):
        V, w = _inputs(nv, length, dtype, seed)
        got = torch.full((nv,), float("nan"), dtype=torch.float64, device="cuda")
        ref = torch.zeros(nv, dtype=torch.float64, device="cuda")
        _noalloc(V, w, got)
        sg.sg_mdot(prob, V, w, ref)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        Vh, wh = V.double().cpu().numpy(), w.double().cpu().numpy()
        bound = np.abs(Vh) @ np.abs(wh)
        m = 11 if dt == "f32" else 4
        assert np.all(np.abs(g - r) <= 2 * m * u * bound), (g, r)
        # the host FP64 product, each sum correctly rounded (math.fsum; FP32
        # inputs multiply exactly in FP64): the device result may differ by
        # the rounding of its summation tree, whose depth is at most the
        # elements one thread adds, plus the block and last-block reductions
        exact = np.array([math.fsum(Vh[i] * wh) for i in range(nv)])
        depth = 11 if dt == "f32" else -(-length // (304 * 256)) + 8 + 304
        assert np.all(np.abs(g - exact) <= 2 * depth * u * bound + U64 * np.abs(exact)), (g, exact)
    prob.close()


def test_noalloc_rejects_too_many_vectors(gpu):
    import torch
    from paper_2310_14649_gb300 import _lib
    V, w = _inputs(33, 16, torch.float64, 3)
    out = torch.zeros(33, dtype=torch.float64, device="cuda")
    st = _lib.lib().sg_mdot_noalloc(0, ctypes.c_void_p(V.data_ptr()), V.stride(0), 33, ctypes.c_void_p(w.data_ptr()),
                                    16, ctypes.c_void_p(out.data_ptr()), None)
    assert st == -1 and b"[1, 32]" in _lib.lib().sg_last_error()

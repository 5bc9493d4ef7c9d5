"""The C-ABI library loads on a machine without a GPU and exports every
entry point declared in include/*.h (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:sg_status|const\s+char\s*\*|void|int|int64_t)\s+\**\s*(sg_\w+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libsg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_14649_gb300 import _lib
    return _lib.lib()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ["sg_setup", "sg_destroy", "sg_apply", "sg_last_error"]:
        assert must in names


def test_exports_every_declared_symbol(libsg):
    missing = [n for n in declared_symbols() if not hasattr(libsg, n)]
    assert not missing, missing


def test_binding_covers_header(libsg):
    from paper_2310_14649_gb300 import _lib
    names = set(declared_symbols()) - {"sg_last_error"}
    bound = set(_lib.SIGNATURES) | set(_lib.VALUE_FUNCTIONS)
    assert names <= bound, sorted(names - bound)
    assert "sg_cnn_param_count" in names


def test_argument_errors_without_gpu(libsg):
    """Host-side argument checks answer before any device work."""
    from paper_2310_14649_gb300 import _lib
    h = ctypes.c_void_p()
    mesh = _lib.MeshDesc(1)
    kl = _lib.KlDesc(0.3, 0.5, 0.5, 0.0, 2, None)
    st = libsg.sg_setup(ctypes.byref(mesh), ctypes.byref(kl), 2, 4, ctypes.byref(h))
    assert st == -1 and b"N must be" in libsg.sg_last_error()
    assert libsg.sg_apply(None, 0, None, 0, None, 0, None) == -1
    assert libsg.sg_destroy(None) == 0
    assert libsg.sg_set_apply_fp64(None, 0) == -1
    n = ctypes.c_int64(0)
    assert libsg.sg_precond_save(None, None, ctypes.byref(n)) == -1
    assert libsg.sg_precond_load(None, b"x" * 64, 64) == -1
    assert libsg.sg_newton(None, None, 0, ctypes.c_double(1e-8), 10, None, None, None) == -1
    assert libsg.sg_nonlinear_residual(None, None, 0, None, 0, None, 0, None) == -1
    assert libsg.sg_nonlinear_jacobian_apply(None, 0, None, 0, None, 0, None, 0, None) == -1
    assert libsg.sg_apply_fp64_info(None, None, None, None) == -1
    assert libsg.sg_set_refine_residual(None, 0) == -1
    assert libsg.sg_refine_residual_info(None, None, None) == -1
    assert libsg.sg_residual_refine(None, None, 0, None, 0, None, 0, None) == -1
    assert libsg.sg_apply_config(None, 0, 1, 1, 1, 1, 8, 1, 0, 1, 4) == -1


def test_cnn_param_count_without_gpu(libsg):
    """The flat weight array of the learned smoother: 9 Cin Cout + Cout per layer."""
    from paper_2310_14649_gb300 import CNN_CHANNELS, sg_cnn_param_count
    ch = CNN_CHANNELS
    assert sg_cnn_param_count() == sum(9 * ch[l] * ch[l + 1] + ch[l + 1] for l in range(5))

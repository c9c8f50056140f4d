"""The C-ABI library loads on a machine without a GPU, exports every entry
point declared in include/*.h, and rejects bad arguments before touching the
device."""
import ctypes
import glob
import os
import re

import pytest

import paper_1604_06236_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s*(nufft_[a-z0-9_]+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    pkg.build()
    return pkg.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert {"nufft_plan", "nufft_inv4", "nufft_inv5", "nufft_fwd1", "nufft_fwd2", "nufft_destroy"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n


def test_status_strings(L):
    for code, name in enumerate(["NUFFT_OK", "NUFFT_ERR_ARG", "NUFFT_ERR_DUP_NODES", "NUFFT_ERR_ALLOC",
                                 "NUFFT_ERR_CUDA", "NUFFT_ERR_TIMEOUT", "NUFFT_ERR_ACCURACY"]):
        assert L.nufft_status_string(code).decode() == name


def _plan(L, N, xptr, tol, prec):
    h = ctypes.c_void_p()
    st = L.nufft_plan(N, xptr, tol, prec, None, ctypes.byref(h))
    return st, h


def test_argument_errors_without_device(L):
    x = (ctypes.c_double * 4)(0.0, 1.0, 2.0, 3.0)
    xp = ctypes.cast(x, ctypes.c_void_p)
    assert _plan(L, 0, xp, 1e-5, 1)[0] == 1
    assert _plan(L, -3, xp, 1e-5, 1)[0] == 1
    assert _plan(L, 4, None, 1e-5, 1)[0] == 1
    assert _plan(L, 4, xp, 1e-5, 3)[0] == 1
    assert _plan(L, 4, xp, 0.0, 1)[0] == 1
    assert _plan(L, 4, xp, float("nan"), 1)[0] == 1
    assert _plan(L, 4, xp, 0.5, 1)[0] == 1
    assert b"tol" in L.nufft_last_error_message()
    # tolerances the precision cannot reach
    assert _plan(L, 4, xp, 1e-7, 1)[0] == 6
    assert _plan(L, 4, xp, 1e-14, 2)[0] == 6
    assert L.nufft_plan(4, xp, 1e-5, 1, None, None) == 1
    # null plan handles
    assert L.nufft_inv5(None, xp, xp, 1, None) == 1
    assert L.nufft_destroy(None) == 0
    assert L.nufft_plan_info(None, None) == 1
    # the measurement utility checks its arguments before touching a device
    r = ctypes.c_double()
    assert L.nufft_measure_fma(3, ctypes.byref(r), None) == 1
    assert L.nufft_measure_fma(1, None, None) == 1


def test_save_restore_argument_errors_without_device(L):
    x = (ctypes.c_double * 4)(0.0, 1.0, 2.0, 3.0)
    xp = ctypes.cast(x, ctypes.c_void_p)
    h = ctypes.c_void_p()
    L.nufft_plan_save.argtypes = [ctypes.c_void_p] * 4
    L.nufft_plan_restore.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
    assert L.nufft_plan_save(None, xp, xp, None) == 1
    # saved quantities missing
    assert L.nufft_plan_restore(4, xp, 1e-5, 1, None, None, xp, None, ctypes.byref(h)) == 1
    assert L.nufft_plan_restore(4, xp, 1e-5, 1, None, xp, None, None, ctypes.byref(h)) == 1
    # convolution-form plans are not restorable
    assert L.nufft_plan_restore(4, xp, 1e-5, 1 | 0x400, None, xp, xp, None, ctypes.byref(h)) == 1
    assert b"TOEPLITZ" in L.nufft_last_error_message()

"""The plan kernels' table-driven e^{j 2 pi T / 2^64} (exact 64-bit turn count
T) against extended-precision host values, through a test hook of the C
library: every component within 4e-16 (a few float64 ulp)."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402


def _reference(T):
    # long double carries at least 64 mantissa bits (80-bit or IEEE quad), so
    # T / 2^64 is exact and the angle is good to ~1e-19
    pi = np.longdouble("3.141592653589793238462643383279502884197")
    a = 2 * pi * (T.astype(np.longdouble) / np.longdouble(2.0) ** 64)
    return np.cos(a), np.sin(a)


def test_cis_turns_table_accuracy():
    if np.finfo(np.longdouble).nmant < 63:
        pytest.skip("long double lacks 64 mantissa bits on this host")
    g = synth.rng(31)
    edges = [0, 1, (1 << 52) - 1, 1 << 52, (1 << 52) + 1, 1 << 62, 1 << 63, (1 << 63) + 12345,
             (1 << 64) - 1, (1 << 64) - (1 << 52), 4095 << 52, 2048 << 52]
    T = np.concatenate([np.array(edges, dtype=np.uint64), g.integers(0, 2**63, size=4000, dtype=np.uint64) * 2 +
                        g.integers(0, 2, size=4000, dtype=np.uint64)])
    Td = torch.from_numpy(T.view(np.int64)).cuda()
    out = torch.empty(T.size, dtype=torch.complex128, device="cuda")
    L = pkg.lib()
    L.nufft_debug_cis.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    pkg.check(L.nufft_debug_cis(T.size, ctypes.c_void_p(Td.data_ptr()), ctypes.c_void_p(out.data_ptr()), None))
    got = out.cpu().numpy()
    c, s = _reference(T)
    err = max(np.max(np.abs(got.real.astype(np.longdouble) - c)), np.max(np.abs(got.imag.astype(np.longdouble) - s)))
    assert float(err) <= 4e-16, float(err)


def test_dd_exp_accuracy():
    """The double-float exponential of the plan's spreading kernels (Tang's
    table-driven method, double-float reduction) over its range -87 < x <= 0,
    against long-double host values of exp at the double-float input it
    receives: absolute error within 4e-15 (2^-48, the double-float format's
    own precision, is 3.6e-15), relative error within 1e-14 down to
    x = -30 (a few units of the double-float format's 2^-48)."""
    if np.finfo(np.longdouble).nmant < 63:
        pytest.skip("long double lacks 64 mantissa bits on this host")
    g = synth.rng(32)
    ln2_64 = np.log(2.0) / 64
    edges = [0.0, -1e-30, -1e-8, -ln2_64 / 2, -ln2_64, -ln2_64 * 1.5, -np.log(2.0), -1.0, -10.0, -86.9, -30.0]
    x = np.concatenate([np.array(edges), -g.uniform(0, 87.0, 3000), -g.uniform(0, 1.0, 1000),
                        -ln2_64 * np.arange(1, 400) + 1e-17])
    x = np.minimum(x, 0.0)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    L = pkg.lib()
    L.nufft_debug_dd_exp.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    pkg.check(L.nufft_debug_dd_exp(x.size, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()), None))
    got = out.cpu().numpy().astype(np.longdouble)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    x_eff = hi.astype(np.longdouble) + lo.astype(np.longdouble)
    ref = np.exp(x_eff)
    abs_err = np.abs(got - ref)
    assert float(abs_err.max()) <= 4e-15, (float(abs_err.max()), float(x[np.argmax(abs_err)]))
    m = x >= -30
    rel = abs_err[m] / ref[m]
    assert float(rel.max()) <= 1e-14, float(rel.max())


def test_exp64_accuracy():
    """The plan kernels' table-driven float64 exponential (Tang's method, used
    for the magnitude of the kernel samples of Eq. 29) over |x| < 700 against
    long-double host values: relative error within 4 float64 ulp (8.9e-16)."""
    if np.finfo(np.longdouble).nmant < 63:
        pytest.skip("long double lacks 64 mantissa bits on this host")
    g = synth.rng(33)
    ln2_64 = np.log(2.0) / 64
    x = np.concatenate([np.array([0.0, 1e-300, -1e-300, 1e-8, -1e-8, ln2_64 / 2, -ln2_64 / 2, 1.0, -1.0,
                                  699.0, -699.0, 50.0, -50.0]),
                        g.uniform(-700.0, 700.0, 4000), g.uniform(-2.0, 2.0, 2000),
                        ln2_64 * np.arange(-500, 500) + 1e-13])
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    L = pkg.lib()
    L.nufft_debug_exp64.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    pkg.check(L.nufft_debug_exp64(x.size, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()), None))
    got = out.cpu().numpy().astype(np.longdouble)
    ref = np.exp(x.astype(np.longdouble))
    rel = np.abs(got - ref) / ref
    assert float(rel.max()) <= 8.9e-16, (float(rel.max()), float(x[np.argmax(rel)]))

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

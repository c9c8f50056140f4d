"""The allocation-free type-5 entry point, nufft_inv5_noalloc.

Callers that cannot allocate device memory while they transform (real-time
loops or embedded runtimes that forbid allocation after set-up, processes
whose device memory comes from an external allocator under a fixed budget)
use nufft_inv5_noalloc, which runs on a fixed scratch array inside the
library instead of taking memory per call.  These checks call it through the
C ABI twice in a row and compare each result with nufft_inv5 on the same
input, within the inverse-transform tolerances of the parity suite.  The file
is collected last, so a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402

TOL = {pkg.FP32: 1e-5, pkg.FP64: 1e-10}
DT = {pkg.FP32: torch.complex64, pkg.FP64: torch.complex128}


def _lib():
    pkg.build()
    L = pkg.lib()
    L.nufft_inv5_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p]
    L.nufft_inv5_noalloc.restype = ctypes.c_int
    return L


def _rel(a, b):
    return float((torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item())


@pytest.mark.parametrize("prec,N", [(pkg.FP32, 4096), (pkg.FP64, 1000), (pkg.FP32, 65536), (pkg.FP64, 65536)])
def test_noalloc_matches_inv5_twice(prec, N):
    L = _lib()
    x = torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=N + 5)).cuda()
    plan = pkg.Plan(x, prec=prec)
    stream = torch.cuda.current_stream()
    for call in range(2):
        f = torch.from_numpy(synth.cn01((3, N), seed=100 * call + N)).to(DT[prec]).cuda()
        ref = plan.inv5(f)
        out = torch.empty_like(f)
        st = L.nufft_inv5_noalloc(plan._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), 3,
                                  ctypes.c_void_p(stream.cuda_stream))
        pkg.check(st)
        torch.cuda.synchronize()
        assert _rel(out, ref) <= TOL[prec], (call, _rel(out, ref))


def test_noalloc_rejects_oversized_plans_and_host_buffers():
    L = _lib()
    N = 1 << 19
    plan = pkg.Plan(torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=3)).cuda(), prec=pkg.FP32)
    f = torch.zeros(N, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(f)
    st = L.nufft_inv5_noalloc(plan._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1, None)
    assert st == 1
    assert b"static scratch" in L.nufft_last_error_message()
    small = pkg.Plan(torch.from_numpy(synth.jittered_nodes(256, 0.45, seed=4)).cuda(), prec=pkg.FP32)
    fh = torch.zeros(256, dtype=torch.complex64)
    oh = torch.empty_like(fh)
    st = L.nufft_inv5_noalloc(small._h, ctypes.c_void_p(fh.data_ptr()), ctypes.c_void_p(oh.data_ptr()), 1, None)
    assert st == 1

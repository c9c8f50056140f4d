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


# (precision, flags, N): default, convolution-form (TOEPLITZ) and refined
# (REFINE) plans, power-of-two and Bluestein N, and the largest power-of-two N
# the 8 MiB array holds for each kind of plan
CASES = [
    (pkg.FP32, 0, 4096), (pkg.FP64, 0, 1000), (pkg.FP32, 0, 65536), (pkg.FP64, 0, 65536),
    (pkg.FP32, 0, 131072),
    (pkg.FP32, pkg.TOEPLITZ, 4096), (pkg.FP64, pkg.TOEPLITZ, 1009),
    (pkg.FP32, pkg.REFINE, 1000), (pkg.FP64, pkg.REFINE, 4096),
    (pkg.FP32, pkg.REFINE, 65536), (pkg.FP64, pkg.REFINE, 32768),
]


@pytest.mark.parametrize("prec,flags,N", CASES)
def test_noalloc_matches_inv5_twice(prec, flags, N):
    L = _lib()
    x = torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=N + 5)).cuda()
    plan = pkg.Plan(x, prec=prec | flags)
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


def test_noalloc_refined_plan_is_refined():
    """On clustered nodes (1% within 0.01-0.05 grid spacings of a neighbour)
    the refined no-alloc result meets the tolerance against Gaussian
    elimination and is closer to it than the unrefined one: the refinement
    is not dropped."""
    import oracle
    oracle.build()
    N = 4096
    xn = synth.clustered_nodes(N, 0.45, 0.01, 0.01, 0.05, seed=21)
    f = synth.cn01(N, seed=22).astype(np.complex64)
    cr = oracle.inv5(xn, f.astype(complex))
    x = torch.from_numpy(xn).cuda()
    ft = torch.from_numpy(f).cuda()
    L = _lib()
    errs = {}
    for name, flags in (("plain", 0), ("refined", pkg.REFINE)):
        plan = pkg.Plan(x, prec=pkg.FP32 | flags)
        out = torch.empty_like(ft)
        pkg.check(L.nufft_inv5_noalloc(plan._h, ctypes.c_void_p(ft.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        torch.cuda.synchronize()
        errs[name] = oracle.rel_l2(out.cpu().numpy().astype(complex), cr)
    assert errs["refined"] <= TOL[pkg.FP32], errs
    assert errs["refined"] < errs["plain"], errs


def test_noalloc_rejects_oversized_plans_and_host_buffers():
    L = _lib()
    N = 1 << 19
    plan = pkg.Plan(torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=3)).cuda(), prec=pkg.FP32)
    f = torch.zeros(N, dtype=torch.complex64, device="cuda")
    out = torch.empty_like(f)
    st = L.nufft_inv5_noalloc(plan._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1, None)
    assert st == 1
    assert b"static scratch" in L.nufft_last_error_message()
    # one size step above the refined limits
    for prec, N in ((pkg.FP32, 131072), (pkg.FP64, 65536)):
        big = pkg.Plan(torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=5)).cuda(), prec=prec | pkg.REFINE)
        fb = torch.zeros(N, dtype=DT[prec], device="cuda")
        ob = torch.empty_like(fb)
        st = L.nufft_inv5_noalloc(big._h, ctypes.c_void_p(fb.data_ptr()), ctypes.c_void_p(ob.data_ptr()), 1, None)
        assert st == 1, (prec, N)
        assert b"(refined)" in L.nufft_last_error_message()
    small = pkg.Plan(torch.from_numpy(synth.jittered_nodes(256, 0.45, seed=4)).cuda(), prec=pkg.FP32)
    fh = torch.zeros(256, dtype=torch.complex64)
    oh = torch.empty_like(fh)
    st = L.nufft_inv5_noalloc(small._h, ctypes.c_void_p(fh.data_ptr()), ctypes.c_void_p(oh.data_ptr()), 1, None)
    assert st == 1

"""Failure detection without a GPU fault: a bounded in-kernel wait on a
barrier phase that nothing completes gives up (after about a second, the
limit the TMA-fed FFT passes use), the host reads NUFFT_ERR_TIMEOUT from
nufft_stream_check, the count is cleared, and the context stays usable."""
import ctypes
import time

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402


def test_expired_wait_is_reported_and_the_context_stays_usable():
    L = pkg.lib()
    L.nufft_debug_wait_expiry.argtypes = [ctypes.c_void_p]
    L.nufft_debug_wait_expiry.restype = ctypes.c_int
    pkg.stream_check()                       # nothing pending
    t0 = time.perf_counter()
    assert L.nufft_debug_wait_expiry(None) == 0
    with pytest.raises(pkg.NufftError) as err:
        pkg.stream_check()
    assert err.value.status == "NUFFT_ERR_TIMEOUT"
    assert time.perf_counter() - t0 < 30.0   # the wait gave up by its time limit
    pkg.stream_check()                       # the count was cleared
    # the library and the context still work: a TMA-fed FFT and a plan + inverse
    n, batch = 65536, 8
    x = synth.cn01((batch, n), seed=5)
    buf = torch.from_numpy(x).to(torch.complex64).cuda().contiguous()
    L.nufft_debug_fft.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p]
    pkg.check(L.nufft_debug_fft(n, 1, -1, batch, ctypes.c_void_p(buf.data_ptr()), None))
    got = buf.cpu().numpy().astype(np.complex128)
    ref = np.fft.fft(x.astype(np.complex64).astype(np.complex128), axis=1)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 3e-6
    pkg.stream_check()

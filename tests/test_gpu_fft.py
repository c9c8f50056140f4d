"""The library's FFT (Stockham passes, power-of-two kernels, mixed radix,
Bluestein) against numpy's FFT, through a test hook of the C library."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402

SIZES = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384, 65536, 131072, 1 << 18,
         1 << 20, 1 << 21, 3, 5, 6, 7, 12, 100, 1000, 1536, 6000, 40960, 655360, 11, 17, 1009, 4099]


def _run(n, prec, dir_, x):
    L = pkg.lib()
    L.nufft_debug_fft.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p]
    dt = torch.complex64 if prec == 1 else torch.complex128   # prec 3 converts in place
    buf = torch.from_numpy(x).to(dt).cuda().contiguous()
    pkg.check(L.nufft_debug_fft(n, prec, dir_, x.shape[0], ctypes.c_void_p(buf.data_ptr()), None))
    return buf.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n", SIZES)
def test_fft_matches_numpy(n, prec):
    batch = 3 if n <= (1 << 18) else 1
    x = synth.cn01((batch, n), seed=n)
    xr = x.astype(np.complex64).astype(np.complex128) if prec == 1 else x
    tol = 2e-6 if prec == 1 else 1e-13
    for dir_ in (-1, 1):
        ref = np.fft.fft(xr, axis=1) if dir_ < 0 else np.fft.ifft(xr, axis=1) * n
        got = _run(n, prec, dir_, x)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < tol * max(1.0, np.log2(max(n, 2)) / 10), (n, prec, dir_, err)


@pytest.mark.parametrize("n,batch", [(8, 2), (256, 2), (2048, 1), (4096, 2), (65536, 1), (65536, 3), (131072, 3),
                                     (1 << 20, 1), (1 << 21, 1), (65536, 40), (1000, 2), (1009, 2), (40960, 2)])
def test_double_float_fft_matches_numpy(n, batch):
    """The double-float FFT (prec 3: pairs of float32) on float64 data reaches
    float64-class accuracy: power-of-two lengths from 2^11 on few vectors run
    the shared-memory radix-4 passes (two or three passes of radix 2^5..2^10),
    larger batches the radix-64 streaming passes, other lengths the general
    passes or Bluestein."""
    x = synth.cn01((batch, n), seed=n + batch)
    for dir_ in (-1, 1):
        ref = np.fft.fft(x, axis=1) if dir_ < 0 else np.fft.ifft(x, axis=1) * n
        got = _run(n, 3, dir_, x)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 2e-13, (n, dir_, err)


@pytest.mark.parametrize("n,batch", [(65536, 64), (131072, 40), (1 << 18, 9), (32768, 70)])
def test_tma_fed_passes_many_tiles(n, batch):
    """float32 power-of-two plans whose radix-256/512 passes run on the
    TMA-fed persistent kernel, with batches large enough that every CTA walks
    several tiles through its ring of stages (32768 = 256 x 128 mixes it with
    the register-loading pass)."""
    x = synth.cn01((batch, n), seed=n + batch)
    xr = x.astype(np.complex64).astype(np.complex128)
    for dir_ in (-1, 1):
        ref = np.fft.fft(xr, axis=1) if dir_ < 0 else np.fft.ifft(xr, axis=1) * n
        got = _run(n, 1, dir_, x)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 3e-6, (n, batch, dir_, err)
    pkg.stream_check()   # no bounded wait gave up

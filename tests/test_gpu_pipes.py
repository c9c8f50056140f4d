"""The measurement utility nufft_measure_fma: finite, positive FMA rates, the
float64 rate below the float32 rate, and argument errors."""
import ctypes
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402


def test_fma_rates_are_ordered():
    f32 = pkg.measure_fma(pkg.FP32)
    f64 = pkg.measure_fma(pkg.FP64)
    assert math.isfinite(f32) and math.isfinite(f64)
    assert f32 > 1.0, f32           # TFLOP/s
    assert 0.0 < f64 < f32, (f64, f32)


def test_fma_rate_rejects_bad_arguments():
    L = pkg.lib()
    r = ctypes.c_double()
    assert L.nufft_measure_fma(3, ctypes.byref(r), None) != 0
    assert L.nufft_measure_fma(pkg.FP32, None, None) != 0

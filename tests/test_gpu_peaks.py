"""The measured arithmetic rates that the rooflines divide by: FP32 FMA
chains (scalar and packed f32x2) and FP64 FMA chains on every SM.  The
values are checked for plausibility only (positive, within a wide band
around the GPU's unit counts), and the argument checks for their errors."""
import pytest

from paper_1803_04120_gb300 import sj

pytestmark = pytest.mark.gpu


def test_fma_rates_are_plausible():
    sc, sc_ms = sj.sj_fp32_fma_rate(0, packed=False)
    pk, pk_ms = sj.sj_fp32_fma_rate(0, packed=True)
    f64, f64_ms = sj.sj_fp64_fma_rate(0)
    for v, ms in ((sc, sc_ms), (pk, pk_ms), (f64, f64_ms)):
        assert v > 0 and ms > 0
    # 152 SMs x 128 FP32 lanes x 2 FLOPs x ~2 GHz is about 80 TFLOP/s
    assert 10.0 < sc < 200.0 and 10.0 < pk < 200.0
    # packed instructions halve the issue slots but do not double the rate
    assert 0.5 < pk / sc < 2.5
    assert 0.05 < f64 < 20.0 and f64 < sc


def test_fma_rate_argument_errors():
    lib = sj.load()
    import ctypes
    tf, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.sj_fp64_fma_rate(-1, ctypes.byref(tf), ctypes.byref(ms)) == sj.SJ_EINVAL
    assert lib.sj_fp64_fma_rate(0, None, ctypes.byref(ms)) == sj.SJ_EINVAL
    assert lib.sj_fp32_fma_rate(0, 1, ctypes.byref(tf), None) == sj.SJ_EINVAL

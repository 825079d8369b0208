"""The measured FMA issue rate (burgers_fma_peak) against the figure derived
from the device's SM count, FP32 lanes per SM and its maximum clock."""
import pytest

from paper_2601_12204_b300 import _lib as L

pytestmark = pytest.mark.gpu


def test_fma_peak_is_plausible():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_12204_b300.api import Context
    ctx = Context(0)
    try:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        derived = sms * 128 * 2.032e9  # lane-FMA/s at the maximum SM clock
        f32 = ctx.fma_peak(L.BURGERS_F32)
        f64 = ctx.fma_peak(L.BURGERS_F64)
        # a loaded GPU may clock below its maximum, never run above it
        assert 0.3 * derived < f32 < 1.05 * derived
        assert 0.0 < f64 < f32
        with pytest.raises(Exception):
            ctx.fma_peak(7)
    finally:
        ctx.close()

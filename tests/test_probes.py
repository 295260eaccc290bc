"""The library's own ceilings (qmcspl_probe_cache, qmcspl_probe_fma): positive rates in a sane
order -- L1 above L2, both above zero -- the clock they ran at, and an FP32 multiply-add rate of the
order of 128 per SM clock, packed or not."""
import ctypes

import pytest

from gpu_helpers import dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _probe(fn, arg):
    from paper_1309_6250_gb300 import _lib
    lib = _lib.load()
    a, b, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(dev()):
        _lib.check(getattr(lib, fn)(arg, ctypes.byref(a), ctypes.byref(b), ctypes.byref(m),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return a.value, b.value, m.value


def test_cache_and_fma_probes():
    l1, l1_clk, mhz1 = _probe("qmcspl_probe_cache", 1)
    l2, l2_clk, mhz2 = _probe("qmcspl_probe_cache", 2)
    assert l1 > l2 > 0.0 and l1_clk > l2_clk > 0.0
    for mhz in (mhz1, mhz2):
        assert 300.0 < mhz < 4000.0
    sms = torch.cuda.get_device_properties(dev()).multi_processor_count
    for packed in (0, 1):
        tflops, per_clk, mhz = _probe("qmcspl_probe_fma", packed)
        assert 300.0 < mhz < 4000.0
        # 2 FLOPs per multiply-add; consistent with the reported clock and SM count
        assert tflops == pytest.approx(per_clk * sms * mhz * 1e6 / 1e12, rel=1e-6)
        assert 64.0 <= per_clk <= 1100.0

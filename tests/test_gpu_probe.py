"""The library's ALU probe (mhd_alu_probe), the measured denominator of the
advance's roofline: it runs, and its FP32 and FP64 multiply-add rates lie
within a factor of two of the unit counts of the device at 1-2.1 GHz."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_alu_probe_rates():
    from paper_1112_1710_gb300 import _build, capi
    _build.build()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f32, ms32 = capi.mhd_alu_probe("f32", 16384)
    f64, ms64 = capi.mhd_alu_probe("f64", 256)
    assert ms32 > 0 and ms64 > 0
    lo32, hi32 = sms * 128 * 2 * 1.0e9 / 1e12 / 2, sms * 128 * 2 * 2.1e9 / 1e12 * 1.05
    assert lo32 <= f32 <= hi32, (f32, lo32, hi32)
    assert f64 > 0.0 and f64 < f32, (f64, f32)
    with pytest.raises(Exception):
        capi.mhd_alu_probe("f32", 0)

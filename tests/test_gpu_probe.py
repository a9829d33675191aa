"""The FMA probe behind the ALU rooflines (mdk_fma_peak): the FP32 and FP64
FMA rates of the device, each within a factor of two of what the SM count
and clock allow (152 SMs x 128 FP32 lanes x 2 FLOP x ~2 GHz = ~80 TFLOP/s;
FP64 at GB300's nominal 1.25 TFLOP/s), and FP32 well above FP64."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_peaks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22951_gb300 import _build, mdk
    _build.build()
    mdk.load()
    f32 = mdk.fma_peak("mixed")
    f64 = mdk.fma_peak("fp64")
    assert 40.0 < f32 < 160.0, f32
    assert 0.6 < f64 < 2.5, f64
    assert f32 > 10 * f64
    with pytest.raises(mdk.MDKError):
        mdk._check(mdk.load().mdk_fma_peak(7, None), "mdk_fma_peak")

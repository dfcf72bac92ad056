"""The peak probes behind the roofline denominators: the measured FP32 FMA
rate lies between half and 110 % of the rate derived from the device's SM
count and maximum clock (128 FP32 lanes per SM, 2 flops per FMA); packed
FP32x2 FMAs are measured at most 10 % above the scalar rate (two lanes per
instruction, the same FMA-pipe time); FP64 runs at a small fraction of FP32."""
import subprocess

import pytest
import torch

from paper_2507_11289_gb300 import dsea

pytestmark = pytest.mark.gpu


def _max_sm_mhz():
    out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=clocks.max.sm",
                          "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20).stdout
    return float(out.strip().splitlines()[0])


def test_probe_rates_are_physical():
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    derived = sms * 128 * 2 * _max_sm_mhz() * 1e6 / 1e12
    f32 = dsea.probe_peak(dsea.PROBE_FP32)
    f32x2 = dsea.probe_peak(dsea.PROBE_FP32X2)
    f64 = dsea.probe_peak(dsea.PROBE_FP64)
    print(f"FP32 {f32:.1f}, FP32x2 {f32x2:.1f}, FP64 {f64:.2f} TFLOP/s; derived FP32 {derived:.1f}")
    assert 0.5 * derived <= f32 <= 1.1 * derived
    assert f32x2 <= 1.1 * f32
    assert 0.0 < f64 < 0.25 * f32
    with pytest.raises(dsea.DseaError):
        dsea.probe_peak(7)

"""The measured CUDA-core peaks (smr_measure_peak) that the CUDA-core
roofline is taken against: each within a plausible band of GB300's unit
counts times its clock (152 SMs; 128 FP32 lanes, 2 FP64 FMA per SM and
clock at up to 2.07 GHz), and an unknown kind refused."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2407_21724_gb300 import smr

FP32_NOMINAL = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_NOMINAL = 152 * 2 * 2 * 2.07e9 / 1e12


def test_measured_peaks():
    torch.cuda.init()
    f32 = smr.smr_measure_peak(0)
    f32x2 = smr.smr_measure_peak(1)
    f64 = smr.smr_measure_peak(2)
    assert 0.3 * FP32_NOMINAL < max(f32, f32x2) < 2.1 * FP32_NOMINAL, (f32, f32x2)
    assert 0.3 * FP64_NOMINAL < f64 < 1.5 * FP64_NOMINAL, f64
    with pytest.raises(smr.SmrError):
        smr.smr_measure_peak(3)

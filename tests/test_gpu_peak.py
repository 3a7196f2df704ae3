"""The measured FP32 FFMA rate (the second denominator of the interaction
kernels' roofline) through the C ABI: it must be positive and may not exceed
the rate the hardware can issue (SM count x 128 lanes x 2 flops x the maximum
SM clock) by more than timing noise."""
import pytest

from paper_1606_02738_gb300 import sph

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_within_the_issue_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    props = torch.cuda.get_device_properties(0)
    r = sph.sph_fp32_peak(0)
    assert r["ms"] > 0
    # no clock query here: 2.2 GHz bounds every GB300 SM clock from above
    limit = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    assert 0.2 * limit < r["tflops"] <= 1.02 * limit, (r, limit)


def test_fp32_peak_rejects_a_bad_device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pytest.raises(sph.SphError) as e:
        sph.sph_fp32_peak(torch.cuda.device_count() + 3)
    assert e.value.code == sph.SPH_EINVAL

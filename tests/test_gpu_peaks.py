"""The arithmetic-peak probe (the denominator of the FP64 path's arithmetic roofline)."""
import pytest

from paper_2307_16758_gb300 import build as B
from paper_2307_16758_gb300 import swe

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    swe.load_library()


def test_fma_peaks_are_plausible_and_fp64_is_the_slow_unit():
    import torch
    props = torch.cuda.get_device_properties(0)
    fp32 = swe.swe_fma_peak("fp32")
    fp64 = swe.swe_fma_peak("fp64")
    # at most what 128 FP32 / 64 FP64 FMA lanes per SM could give at 3 GHz
    assert 0 < fp32 <= 2 * 128 * props.multi_processor_count * 3e9
    assert 0 < fp64 <= 2 * 64 * props.multi_processor_count * 3e9
    assert fp32 > 4 * fp64

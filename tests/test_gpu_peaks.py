"""The measured FP32 and ex2 throughput (pm_measure_peaks) that the roofline
fractions divide by: positive, at most what the SM count, the 128 FP32 lanes
per SM and the maximum clock allow, and at least half of it (an FFMA-only
kernel at full occupancy that reached less would not be a peak)."""
import pytest
import torch

import paper_2411_01919_b300 as pm

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    m = pm.measure_peaks()
    props = torch.cuda.get_device_properties(0)
    assert m['sm_count'] == props.multi_processor_count
    max_ghz = 2.2                          # above any B300 SM clock
    derived_max = m['sm_count'] * 128 * 2 * max_ghz / 1e3
    assert 0.5 * m['sm_count'] * 128 * 2 * 1.0 / 1e3 < m['fp32_tflops'] <= derived_max
    # the special-function unit is far narrower than the FMA pipes
    assert 0.0 < m['ex2_tops'] < m['fp32_tflops'] / 2
    print('measured: %.1f TFLOP/s FP32, %.2f Tex2/s, %d SMs'
          % (m['fp32_tflops'], m['ex2_tops'], m['sm_count']))

"""The measured peaks the roofline is quoted against: the integer-ALU rate (lop3 and
multiply-add) and the shared-memory load bandwidth, checked against the device's own counts
(SMs x lanes or bytes per clock x a clock between 1 and 2.2 GHz)."""
import pytest
import torch

import paper_2509_23043_gb300 as pt

pytestmark = pytest.mark.gpu


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_integer_pipe_rates_are_within_the_lane_counts():
    sms = _sms()
    for kind in (0, 1):
        ops, ms = pt.calibrate_int(kind)
        assert ms > 0
        # at most 64 (ALU) or 64 (multiply) lanes per SM per clock, at most 2.2 GHz
        assert 0.25 * sms * 64 * 1.0e9 < ops < sms * 64 * 2.2e9 * 1.01, (kind, ops)
    with pytest.raises(pt.PTError):
        pt.calibrate_int(2)


def test_shared_memory_bandwidth_is_within_the_bank_width():
    sms = _sms()
    bps, ms = pt.calibrate_smem()
    assert ms > 0
    # 32 banks x 4 B is 128 B per clock per SM; allow up to twice that, at most 2.2 GHz
    assert sms * 64 * 1.0e9 < bps < sms * 256 * 2.2e9 * 1.01, bps

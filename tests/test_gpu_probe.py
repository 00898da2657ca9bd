"""The FP32 rate probe that the ALU rooflines divide by: both forms run on
every lane of every SM and land near the nominal rate (SMs x 128 lanes x
clock), and bad arguments are refused."""
import pytest

from paper_2602_19873_gb300 import nl

pytestmark = pytest.mark.gpu


def test_fp32_rate_near_nominal():
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    clock_ghz = 2.07   # the GB300's highest SM clock; the probe may run below it
    nominal = sms * 128 * clock_ghz * 1e9
    for packed in (False, True):
        ops, ms = nl.probe_fp32_rate(packed, 3)
        assert ms > 0.0
        assert 0.3 * nominal < ops < 1.1 * nominal, (packed, ops / nominal)


def test_fp32_rate_rejects_bad_reps():
    with pytest.raises(nl.NLError) as e:
        nl.probe_fp32_rate(False, 0)
    assert e.value.status == 1

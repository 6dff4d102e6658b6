"""The bench's clock record (nvidia-smi samples taken during the timed region),
checked on the CPU with sample lines in nvidia-smi's csv,noheader,nounits form:
the median SM clock under load, the maximum clock, every throttle reason seen
active at least once, and lines that are not samples skipped."""
import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_median_max_and_reasons():
    lines = ["0, 2070, 2070, 410.5, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 905.0, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 880.2, Not Active, Not Active, Not Active, Not Active",
             "garbage",
             "0, [N/A], 2070, 1.0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 990.1, Active, Not Active, Not Active, Not Active"]
    out = _sampler(lines).summary()
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2062.5 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_no_samples():
    out = _sampler([]).summary()
    assert out == dict(sm_mhz=None, sm_max_mhz=None, reasons=[], samples=0)

"""bench.py's host-side contract pieces, on the CPU: the metric string, the
defaults keep >= 3 warm-up steps, and the clock sampler's summary (median SM
clock, throttle reasons) reads nvidia-smi's CSV."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_metric_and_defaults():
    b = _bench()
    assert "Mpix/s" in b.METRIC and "1080p" in b.METRIC
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = b.parse_args()
    finally:
        sys.argv = argv
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"


def test_clock_summary_median_and_reasons(tmp_path):
    b = _bench()
    cs = b.ClockSampler(0)
    cs.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 510.2, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 540.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 530.5, 0x0, Not Active, Not Active, Not Active, Not Active"]
    open(cs.path, "w").write("\n".join(rows) + "\n")
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and s["power_w_max"] == 540.0
    assert not os.path.exists(cs.path)  # the temporary CSV is removed


def test_clock_summary_without_nvidia_smi(tmp_path):
    b = _bench()
    cs = b.ClockSampler(0)
    cs.path = str(tmp_path / "missing.csv")
    s = cs.summary()
    assert s["samples"] == 0 and s["reasons"] == ["nvidia-smi unavailable"]

"""bench.py's host-side contract pieces, on the CPU: the metric string, the
defaults keep >= 3 warm-up steps, the clock sampler's summary (median SM
clock, throttle reasons) reads nvidia-smi's CSV, and the reference arm (the
CPU oracle) prints its JSON line on rank 0 only."""
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


def _run_bench(args, env_extra=None, timeout=600):
    import subprocess
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_the_contract_line():
    """The reference arm times the CPU oracle on a bounded sample of the
    1080p workload and prints one JSON line on the same metric, with its
    cpu_baseline and an e2e block that moves no bytes across the host link."""
    import json
    b = _bench()
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == b.METRIC and line["unit"] == "Mpix/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert abs(line["ms_per_step"] - 1920 * 1080 / line["value"] / 1e3) < 1e-2 * line["ms_per_step"]


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""

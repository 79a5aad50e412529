"""bench.py's contract on the CPU: the reference arm (the FP64 oracle timed on the host cores) prints one
JSON line with the keys the contract names, other ranks print nothing, workloads it does not cover get an
`unavailable` line; the clock-sampler summary reads nvidia-smi's CSV (median SM clock, throttle
reasons) correctly; and the key of the measured-traffic table follows the kernel's code, not its comments."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env_extra=None, timeout=300):
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          cwd=ROOT, env=env, timeout=timeout)


def test_reference_arm_prints_the_contract_line():
    out = _bench("--impl", "reference", "--workload", "single256", "--steps", "1", "--warmup", "1")
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == d["unit"] == "Gcell-updates/s" and d["value"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1 and d["ms_per_step"] > 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["config"]["workload"] == "single256"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_are_silent():
    out = _bench("--impl", "reference", "--workload", "single256", "--steps", "1", "--warmup", "1",
                 env_extra={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_reference_arm_unavailable_for_batches():
    out = _bench("--impl", "reference", "--workload", "batch256", "--steps", "1", "--warmup", "1")
    assert out.returncode == 0
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and "unavailable" in d


def test_clock_summary(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    p = tmp_path / "clocks.csv"
    rows = [
        "0, 1980, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1190.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1201.3, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    p.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler(0, str(p)).summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    p.write_text("0, 1500, 2070, 1300.0, 0x0000000000000048, Active, Not Active, Active, Not Active\n")
    s = bench.ClockSampler(0, str(p)).summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1500.0
    p.write_text("")
    assert bench.ClockSampler(0, str(p)).summary()["reasons"] == ["no samples"]


def test_traffic_key_ignores_comments():
    """The measured DRAM traffic is keyed on the kernel's code, not its comments or layout."""
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) {  // add one\n    return x + 1; /* the\n result */ }\n"
    b = "// header\nint f(int x) {\n  return x + 1;\n}\n"
    assert bench.code_only(a) == bench.code_only(b) == "int f(int x) { return x + 1; }"
    assert bench.code_only("return x + 2;") != bench.code_only("return x + 1;")

"""The benchmark's reference arm (the CPU oracle timed on the host cores on a
bounded sample of the headline workload) runs without a GPU and prints one
JSON line with the keys the benchmark contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "Gb/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "D=512" in line["config"]["workload"] and line["config"]["L"] == 42


def test_roofline_bookkeeping():
    """The DRAM traffic record is reported only for the kernel configuration
    and device sources it was captured with, and the roofline arithmetic
    matches the documented formulas."""
    sys.path.insert(0, ROOT)
    import bench
    key, rec = next(iter(bench.PROFILED_TRAFFIC.items()))
    if rec["sources"] == bench.kernel_sources_hash():
        assert bench.profiled_traffic(key) == rec["bytes"]
    assert bench.profiled_traffic((key[0] * 2, key[1], key[2])) is None
    saved = rec["sources"]
    try:
        rec["sources"] = "0" * 16
        assert bench.profiled_traffic(key) is None
    finally:
        rec["sources"] = saved
    # 3N integer operations per state and stage, times the overlap (D + 2L) / D
    assert abs(bench.algorithmic_ops_per_bit(64, 512, 42) - 223.5) < 1e-9
    assert abs(bench.algorithmic_ops_per_bit(256, 1024, 64) - 864.0) < 1e-9
    # 152 SMs x 4 schedulers x 32 lanes x 2 (16x2) x 2.07 GHz
    assert abs(bench.peak_int16_ops(152, 2.07e9) - 80.54784e12) < 1e6

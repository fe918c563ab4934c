"""bench.py --impl reference (the FP64 oracle timed on the host cores) prints
one JSON line with the contract's keys; runs on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--cpu-seconds", "0.2"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GFLOP/s"
    assert d["steps"] == 1 and d["warmup"] == 0 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"]


def test_traffic_capture_matches_the_kernel_sources():
    """roofline.traffic comes from an ncu capture stored with a hash of the
    tcgen05 kernel's sources; it must list the same sources as bench.py and
    match their committed contents, so that an edited kernel without a fresh
    capture shows up here rather than as a null traffic figure."""
    sys.path.insert(0, ROOT)
    import bench

    with open(os.path.join(ROOT, "profiles", "k_umma_traffic.json")) as f:
        d = json.load(f)
    assert d["sources"] == bench.UMMA_SOURCES
    assert bench.umma_traffic() == d["dram_bytes_per_launch_mean"] > 0

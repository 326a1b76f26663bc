"""The benchmark's reference arm (the FP64 oracle on every host core) runs on
a CPU and prints one JSON line with the keys of the benchmark contract."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--packets", "800", "--grid", "32"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["unit"] == d["unit"]
    assert "workload" in d["config"]


def test_rooflines_pick_the_binding_bound():
    """The headline roofline is the bound with the larger fraction of its
    peak (the lower packet rate limit); both bounds are reported."""
    sys.path.insert(0, ROOT)
    import bench
    led = {"deposit_steps": 700.0, "locate_steps": 80.0, "peel_steps": 2100.0, "scatterings": 4.0}
    r = bench.trace_rooflines(led, 1.0, 1e-3, 3, 1e9, 1000.0, "measured", "k", 4, None)
    # bytes 4*2880 + 16*700 + 16*15 = 22960 B in 1 us -> 22.96 GB/s of 1000; reductions 715 in 1 us of 1e9/s
    assert abs(r["roofline_hbm"]["achieved"] - 22.96) < 1e-9
    assert abs(r["roofline_atomic"]["achieved"] - 7.15e8) < 1e-3
    assert r["roofline"]["bound"] == "atomics" and r["roofline"]["frac"] == r["roofline_atomic"]["frac"]
    r = bench.trace_rooflines(led, 1.0, 1e-3, 3, 1e12, 10.0, "measured", "k", 4, 30000.0)
    assert r["roofline"]["bound"] == "hbm" and r["roofline"]["traffic"] == 30000.0

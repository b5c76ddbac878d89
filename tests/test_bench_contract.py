"""bench.py's reference arm (the oracle, timed on the host cores) prints one
JSON line with the contract's keys -- checked here without a GPU, since that
arm needs none."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    # the small pile keeps this quick; the large pile takes the same code path
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--workload", "pile_small"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "body-steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "pile_small" and d["config"]["host_threads"] == d["cpu_baseline"]["cores"]


def test_blend_roofline_arithmetic():
    sys.path.insert(0, ROOT)
    import bench
    # 2 steps of 37 MB in 0.02 ms each against a 6800 GB/s peak
    r = bench.blend_roofline([0.02, 0.02], 2 * 37e6, 2, 6800.0, "measured")
    assert abs(r["achieved"] - 37e6 / 0.02e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-12
    assert r["kernel"] == "k_blend" and r["unit"] == "GB/s" and abs(r["avg_launch_ms"] - 0.02) < 1e-12
    assert bench.blend_roofline([], 0.0, 0, 6800.0, "measured") is None
    assert bench.blend_roofline([0.0], 1.0, 1, None, "none") is None

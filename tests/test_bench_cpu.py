"""bench.py's reference arm (the CPU oracle) and its JSON contract, on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--nmol", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "quartets/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_roofline_traffic_is_null_for_changed_or_unknown_kernels():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.traffic_for("jk_class_kernel<(00|00) prims 1111, fp64>", 1) is None
    # a recorded entry is returned only while the kernel sources hash to the recorded value
    label, g = next(iter(bench.TRAFFIC_BYTES))
    got = bench.traffic_for(label, g)
    assert got is None or got == bench.TRAFFIC_BYTES[(label, g)]

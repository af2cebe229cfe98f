"""bench.py's reference arm (the CPU oracle) and its JSON contract, on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--nmol", "3", "--oracle-sample", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
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
    assert bench.traffic_for(7, 1000) is None   # no such tier
    # recorded bytes are used only while the kernel sources hash to the capture's value
    for tier, (per_q, sha) in bench.TRAFFIC_CAPTURES.items():
        got = bench.traffic_for(tier, 1000)
        if bench.sources_sha() == sha:
            assert got == per_q * 1000
        else:
            assert got is None
        assert bench.traffic_for(tier, 1000, current=False) == per_q * 1000


def test_family_roofline_reports_an_earlier_capture_apart(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    rows = [dict(la=0, lb=0, lc=0, ld=0, na=1, nb=1, nc=1, nd=1, tier=0, threads_per_quartet=1, regs=64,
                 ms=2.0, flops_model=2e9, quartets=100, launches=2)]
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURES", {0: (10.0, "0" * 16)})
    r = bench.family_roofline(rows, 0, None, 2.0)
    assert r["traffic"] is None and r["traffic_note"] is None
    assert r["traffic_earlier_capture"]["bytes_per_launch"] == 500.0
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURES", {0: (10.0, bench.sources_sha())})
    r = bench.family_roofline(rows, 0, None, 2.0)
    assert r["traffic"] == 500.0 and r["traffic_earlier_capture"] is None


def test_family_roofline_arithmetic():
    sys.path.insert(0, ROOT)
    import bench
    rows = [dict(la=1, lb=0, lc=0, ld=0, na=1, nb=3, nc=3, nd=1, tier=0, threads_per_quartet=1, regs=100,
                 ms=2.0, flops_model=2e9, quartets=10, launches=1),
            dict(la=0, lb=0, lc=0, ld=0, na=3, nb=3, nc=3, nd=1, tier=0, threads_per_quartet=1, regs=80,
                 ms=6.0, flops_model=3e9, quartets=30, launches=1),
            dict(la=0, lb=0, lc=0, ld=0, na=3, nb=3, nc=3, nd=1, tier=1, threads_per_quartet=1, regs=60,
                 ms=1.0, flops_model=9e9, quartets=99, launches=1)]
    r = bench.family_roofline(rows, 0, 1.0e12, 10.0)
    assert r["achieved"] == (5e9 / 8e-3) / 1e12 and r["launches"] == 2 and r["launch_ms"] == 4.0
    assert abs(r["frac"] - (5e9 / 8e-3) / bench.PEAK_FP64_NOMINAL) < 1e-15
    assert r["kernel_share"] == 0.8 and r["largest_class"]["class"] == "(00|00)/3331"
    assert bench.family_roofline(rows, 1, None, 10.0)["achieved"] == 9.0

"""bench.py's accelerated-form timing (run_forms) on CPU, against a stand-in
engine: the per-form keys of the JSON line (time, speed-up, deviation from
the base build, quartet split, first-build and compile cost), the option
save/restore around the precision-option forms, and that the base result is
left in J and K. No GPU: CUDA events and synchronisation are replaced by
host stand-ins, and the engine is a Python object with the binding's
methods."""
import os
import sys
import types

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Event:
    clock = 0.0

    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        _Event.clock += 3.0          # every record advances the host clock by 3 ms
        self.t = _Event.clock

    def elapsed_time(self, other):
        return other.t - self.t


class _Engine:
    """The binding's JK methods used by run_forms; each (precision, asym64,
    screen64) combination 'compiles' 5 ms on its first build."""
    h = None

    def __init__(self):
        self.opts = {"compile_ms": 0.0, "asym64": 0.0, "screen64": 1.0, "tau32": 1e-4, "profile": 0.0,
                     "branches": 4.0}
        self.seen = set()
        self.builds = []

    def set_option(self, k, v):
        self.opts[k] = float(v)

    def get_option(self, k):
        return self.opts[k]

    def build(self, Ds, cutoff, precision, J, K, stats):
        key = (precision, self.opts["asym64"], self.opts["screen64"])
        if key not in self.seen:
            self.seen.add(key)
            self.opts["compile_ms"] += 5.0
        self.builds.append((precision, self.opts["tau32"], self.opts["asym64"], self.opts["screen64"]))
        # FP64 build: J = K = 1; every other form off by 1e-9 (J) and 2e-9 (K)
        dj = 0.0 if precision == "fp64" else 1e-9
        for j, k in zip(J, K):
            j.fill_(1.0 + dj)
            k.fill_(1.0 + 2 * dj)
        nq32 = 0 if precision == "fp64" else 75
        return J, K, {"quartets_fp64": 100 - nq32, "quartets_fp32": nq32, "quartets_routed": 0, "ms": 1.0}


def _rows():
    return [dict(la=0, lb=0, lc=0, ld=0, na=1, nb=1, nc=1, nd=1, tier=t, threads_per_quartet=1, regs=64,
                 local_bytes=0, ms=0.5, flops_model=1e6, quartets=50) for t in (0, 1)]


@pytest.fixture
def bench_mod(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2507_09772_gb300 import jk
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(jk, "jk_profile", lambda h: _rows())
    return bench


def test_run_forms_reports_each_form_with_its_first_build_cost(bench_mod):
    eng = _Engine()
    args = types.SimpleNamespace(precision="fp64", forms="fp64,mixed,mixed_asym64,mixed_screen32,mixed@1e-05",
                                 tau32=1e-4, cutoff=1e-13, tune=0, form_steps=2, branches=4, router_margin=0.0)
    Js = [torch.ones(1, 3, 3, dtype=torch.float64)]
    Ks = [torch.ones(1, 3, 3, dtype=torch.float64)]
    flush = torch.empty(16, dtype=torch.uint8)
    out = bench_mod.run_forms(args, eng, [None], [None], Js, Ks, flush, None, base_ms=4.0, base_quartets=100)

    assert set(out) >= {"fp64", "mixed", "mixed_asym64", "mixed_screen32", "mixed@1e-05"}
    assert out["fp64"]["ms_per_step"] == 4.0
    m = out["mixed"]
    # two timed builds between two records 3 ms apart (the events advance the clock once each)
    assert m["ms_per_step"] == pytest.approx(1.5)
    assert m["speedup_vs_fp64"] == pytest.approx(4.0 / 1.5)
    assert m["max_abs_dJ"] == pytest.approx(1e-9, rel=1e-6) and m["max_abs_dK"] == pytest.approx(2e-9, rel=1e-6)
    assert m["within_1e-8"] is True
    assert m["fp32_fraction"] == 0.75 and m["same_quartets_as_fp64"] is True
    assert m["autotune"] is None and m["autotune_s"] >= 0.0
    assert "tiers" in m and "error" not in m["tiers"]
    # first build of each form: compiles once for mixed, once for each precision option, not for a new tau32
    assert m["compile_ms"] == 5.0 and m["first_build_s"] >= 0.0
    assert out["mixed_asym64"]["compile_ms"] == 5.0
    assert out["mixed_screen32"]["compile_ms"] == 5.0
    assert out["mixed@1e-05"]["compile_ms"] == 0.0 and out["mixed@1e-05"]["tau32"] == 1e-5
    assert out["mixed_asym64"]["cost_vs_mixed"] == pytest.approx(0.0)
    # options restored after the option forms
    assert eng.opts["asym64"] == 0.0 and eng.opts["screen64"] == 1.0 and eng.opts["tau32"] == 1e-4
    assert eng.opts["profile"] == 0.0 and eng.opts["branches"] == 4.0
    # the option forms ran with the option set, the tau32 form with its threshold
    assert ("mixed", 1e-4, 1.0, 1.0) in eng.builds and ("mixed", 1e-4, 0.0, 0.0) in eng.builds
    assert ("mixed", 1e-5, 0.0, 1.0) in eng.builds
    # the base (FP64) result is left in J and K
    assert float(Js[0].max()) == 1.0 and float(Ks[0].max()) == 1.0

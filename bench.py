#!/usr/bin/env python
"""Benchmark of the batched direct-SCF JK build on GB300.

Workload (one "step"): J and K of 64 independent seeded molecules of 10-60
atoms (2:1 light:heavy, 6-31G*-shaped Cartesian basis, about 20,000 basis
functions in all), one density each, cutoff 1e-13, all-FP64, every molecule
in the same per-class persistent integral kernels. A step runs the whole
per-iteration path: density block maxima, fused screening + Rys integrals +
contraction with D + atomics (every class pair), symmetrisation of J and K.
Basis setup (pair tables, Schwarz factors) is per geometry and reported as
init_ms, outside the steps.

Metric: significant shell quartets per second (whole job), plus ms per
step. The L2 (129 MB) is flushed before every step by writing a 256 MiB
buffer. Under torchrun each rank builds its own batch of 64 molecules
(weak scaling, no collective on the data path).

--impl reference times the CPU oracle (plain FP64 McMurchie-Davidson) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "JK build ms & quartets/s vs plain FP64 at max|ΔK|≤1e-8; % of FP32/FP64 peak"
UNIT = "quartets/s"
WORKLOAD = "batched-631gs-64mol"
# GB300 FP64: 152 SMs x 4 FLOP/clk/SM (2 FP64 FMA) x 2.07 GHz ~= 1.26 TFLOP/s,
# the 1.25 TFLOP/s nominal figure; FP32: 152 x 256 FLOP/clk x 2.07 GHz.
PEAK_FP64_NOMINAL = 152 * 4 * 2.07e9
PEAK_FP32_NOMINAL = 152 * 256 * 2.07e9

# DRAM traffic of the integral kernel family (dram__bytes_read.sum +
# dram__bytes_write.sum summed over every jk_class_kernel launch of one
# build), from one ncu capture of the 8-molecule case of the batched workload
# (`bench.py --nmol 8 ... --tune 0`, heuristic fragment shapes), per
# significant quartet of that build, per tier; scaled to a step by its quartet
# count. A capture counts as the traffic of the kernels only while the
# kernel sources hash to the value it was taken with; otherwise the roofline
# reports traffic null and gives the capture apart, labelled as earlier.
TRAFFIC_SOURCES = ["paper_2507_09772_gb300/csrc/jk_kernels.cuh", "paper_2507_09772_gb300/csrc/jk_types.h",
                   "paper_2507_09772_gb300/csrc/jk_router.cuh"]
# Captures of the 8-molecule case (profiles/jk_class_kernel_dram_traffic_batched8.md),
# both over 287,529,305 quartets, with the hash of the comment-free kernel
# sources they ran:
#   tier 0 (FP64 build): 1,715,792,896 B read + 3,408,896 B written, on the
#     kernels just before J and K moved from ATOM to RED accumulation;
#   tier 1 (FP32 build): 1,289,914,624 B read + 0 B written, on the RED
#     kernels.
TRAFFIC_CAPTURES = {0: (1719201792 / 287529305, "f7bad00fedd57b74"),
                    1: (1289914624 / 287529305, "83e18b6215b51bc2")}


def sources_sha():
    """Hash of the kernel sources without their comments (the text the
    kernels are compiled from)."""
    import hashlib
    from paper_2507_09772_gb300.build import _strip_comments
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f)) as fh:
            h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def traffic_for(tier, quartets, current=True):
    """DRAM bytes of the class kernels of one tier for `quartets` quartets
    from its capture, or None when there is none. With current (the
    default), None also when the kernel sources have changed since the
    capture."""
    if tier not in TRAFFIC_CAPTURES:
        return None
    per_q, sha = TRAFFIC_CAPTURES[tier]
    if current and sources_sha() != sha:
        return None
    return per_q * quartets


def family_roofline(prof_rows, tier, probe, ms_serial):
    """Roofline of one tier's integral kernels taken as one kernel family
    (every class instantiation of jk_class_kernel): modelled FLOPs of the
    quartets they evaluated over their summed serialised launch times, which
    is the FLOPs per launch over the average launch duration. The work is
    spread over hundreds of class kernels (none above 2 % of the step), so the
    family, not one class, is the dominant kernel."""
    rows = [v for v in prof_rows if v["tier"] == tier]
    if not rows:
        return None
    ms = sum(v["ms"] for v in rows)
    fl = sum(v["flops_model"] for v in rows)
    q = sum(v["quartets"] for v in rows)
    n = sum(v["launches"] for v in rows)
    peak = PEAK_FP64_NOMINAL if tier == 0 else PEAK_FP32_NOMINAL
    ach = fl / (ms * 1e-3) if ms > 0 else 0.0
    dom = max(rows, key=lambda v: v["ms"])
    traffic = traffic_for(tier, q)
    earlier = traffic_for(tier, q, current=False) if traffic is None else None
    return {
        "bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
        "traffic": traffic / n if traffic is not None else None,
        "traffic_note": ("DRAM bytes per launch (family average) from an 8-molecule ncu capture, per quartet, "
                         "scaled by this step's quartets: %.1f GB/s over the launches"
                         % (traffic / (ms * 1e-3) / 1e9)) if traffic is not None else None,
        "traffic_earlier_capture": ({
            "bytes_per_launch": earlier / n, "kernel_sources": TRAFFIC_CAPTURES[tier][1],
            "note": "DRAM bytes per launch from an ncu capture of an earlier version of these kernels (sources "
                    "hash %s, now %s), scaled by this step's quartets; not the traffic of the kernels timed here"
                    % (TRAFFIC_CAPTURES[tier][1], sources_sha())} if earlier is not None else None),
        "kernel": "jk_class_kernel<..., %s> (all %d class instantiations of the tier)"
                  % ("double" if tier == 0 else "float", n),
        "launches": n, "launch_ms": ms / n, "kernel_ms": ms,
        "kernel_share": ms / ms_serial if ms_serial else None,
        "flops_per_launch": fl / n,
        "timing": "CUDA events around each launch, serialised replay after the timed region",
        "peak_source": ("nominal FP64 FMA rate: 152 SMs x 4 FLOP/clk x 2.07 GHz (MEASURED_PEAKS.json has no FP64 "
                        "figure)" if tier == 0 else
                        "nominal FP32 FMA rate: 152 SMs x 256 FLOP/clk x 2.07 GHz (MEASURED_PEAKS.json has no FP32 "
                        "figure)"),
        "peak_probe_tflops": probe / 1e12 if probe else None,
        "frac_of_probe": ach / probe if probe else None,
        "largest_class": {"class": "(%d%d|%d%d)/%d%d%d%d" % (dom["la"], dom["lb"], dom["lc"], dom["ld"], dom["na"],
                                                              dom["nb"], dom["nc"], dom["nd"]),
                          "share_of_tier": dom["ms"] / ms, "tflops_model": dom["flops_model"] / (dom["ms"] * 1e-3) / 1e12,
                          "G": dom["threads_per_quartet"], "regs": dom["regs"]},
    }


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nmol", type=int, default=64)
    ap.add_argument("--workload", default="batch", choices=["batch", "cluster", "highl", "router"],
                    help=("batch: the 64-molecule benchmark (default); cluster: 768-atom water-like "
                          "cluster; highl: 60-atom TZVPP-shaped spherical cluster; router: the "
                          "1,024-atom cluster the router is evaluated on"))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "fp32"])
    ap.add_argument("--cutoff", type=float, default=1e-13)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--oracle-sample", type=int, default=ORACLE_SAMPLE,
                    help="smallest molecules of the batch in the oracle's sample (cpu_baseline and --impl reference)")
    ap.add_argument("--no-probe", action="store_true", help="skip the FMA peak probes (profiling runs)")
    ap.add_argument("--no-forms", action="store_true", help="skip the mixed / routed comparison")
    ap.add_argument("--forms", default="mixed,routed", help="accelerated forms timed against the FP64 build")
    ap.add_argument("--chunk", type=int, default=0, help="candidate kets per work item (0: the library default)")
    ap.add_argument("--router-margin", type=float, default=0.0,
                    help="added to the trained router's margin (log10 units; larger releases fewer quartets)")
    ap.add_argument("--opt", action="append", default=[],
                    help="library option KEY=VALUE set on the handle before the run (repeatable)")
    ap.add_argument("--chunk-fp64tier", type=int, default=0,
                    help="the same for the FP64 tier of mixed and routed builds (0: the library default)")
    ap.add_argument("--oracle-blocks", type=int, default=8,
                    help="single large molecules: J and K shell blocks the oracle computes to check every form")
    ap.add_argument("--form-steps", type=int, default=2)
    ap.add_argument("--tau32", type=float, default=1e-4)
    ap.add_argument("--graph", type=int, default=1, help="replay each build as one CUDA graph")
    ap.add_argument("--branches", type=int, default=4, help="class kernels forked over this many graph branches")
    ap.add_argument("--micro", action="store_true", help="appendix-style micro-benchmarks instead of the workload")
    ap.add_argument("--micro-units", type=int, default=64,
                    help="triatomic units of the d-only / f-only n_dm sweep geometry (3 atoms each)")
    ap.add_argument("--micro-cases", default="ss,d,f,forms",
                    help="micro-benchmark parts: ss ((ss|ss) n_prim sweep), d, f (n_dm sweeps), forms (the rest)")
    ap.add_argument("--tune", type=int, default=1, help="autotune the fragment shapes before the warm-up (untimed)")
    ap.add_argument("--prof-steps", type=int, default=1, help="serialised, per-kernel-timed steps after the timed region")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The CPU oracle's sample of the batched workload, shared by the cpu_baseline
# leg and the --impl reference arm so that both time the same work: the full
# screened FP64 JK of the ORACLE_SAMPLE smallest molecules of the batch.
ORACLE_SAMPLE = 6


def oracle_sample(mols, n=ORACLE_SAMPLE):
    order = sorted(range(len(mols)), key=lambda i: (mols[i].natm, i))
    return [mols[i] for i in order[:n]]


def oracle_pass(sample, cutoff):
    """One pass of the oracle over the sample: (quartets, seconds)."""
    import oracle
    nq = 0
    t0 = time.perf_counter()
    for m in sample:
        _, _, n = oracle.jk(m, cutoff=cutoff)
        nq += n
    return nq, time.perf_counter() - t0


def cpu_oracle_sample(mols, seconds: float, cutoff: float, quartets_per_step=None, nsample=ORACLE_SAMPLE):
    """Oracle (as it stands) on a bounded sample of the workload on the host
    cores. Batched workload: repeated passes over the same molecules the
    reference arm times, until `seconds` pass. A single large molecule: exact
    J shell blocks (row-restricted), sampled until `seconds` pass. The ms of a
    whole step is extrapolated from the rate and labelled so."""
    import numpy as np
    import oracle
    if len(mols) == 1:
        mol = mols[0]
        if mol.spherical:
            # the oracle works in the Cartesian basis: time it on the
            # Cartesian twin with D_cart = C D C^T
            from paper_2507_09772_gb300 import synth
            C = oracle.c2s_matrix(mol)
            sh = mol.shells.copy()
            sh[:, 5] = 0
            mol = synth.Molecule(coords=mol.coords, shells=sh, exps=mol.exps, coeffs=mol.coeffs,
                                 nao=mol.nao_cart, nao_cart=mol.nao_cart,
                                 D=np.stack([C @ d @ C.T for d in mol.D]), name=mol.name + "-cart")
        Q = oracle.schwarz_coulomb(mol)
        rng = np.random.default_rng(0)
        nq, t_total, nb = 0, 0.0, 0
        while t_total < seconds:
            blk = rng.integers(0, mol.nshell, size=(1, 2))
            t0 = time.perf_counter()
            _, _, n = oracle.jk_blocks(mol, blk, np.zeros((0, 2), dtype=np.int32), cutoff=cutoff, Q=Q)
            t_total += time.perf_counter() - t0
            nq += n
            nb += 1
        out = {"value": nq / t_total, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"row-restricted: exact J shell blocks of the molecule ({nb} blocks, {nq} shell "
                         f"quartets, {t_total:.1f} s; each screened quartet of a block counted once)"}
    else:
        sample = oracle_sample(mols, nsample)
        nq, t_total, passes = 0, 0.0, 0
        while t_total < seconds or passes == 0:
            n, dt = oracle_pass(sample, cutoff)
            nq += n
            t_total += dt
            passes += 1
        out = {"value": nq / t_total, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"full screened FP64 JK of the {len(sample)} smallest molecules of the batch "
                         f"({min(m.natm for m in sample)}-{max(m.natm for m in sample)} atoms, "
                         f"{nq // passes} quartets per pass, {passes} passes, {t_total:.1f} s); the same "
                         f"sample as each step of --impl reference"}
    if quartets_per_step:
        out["extrapolated_ms_per_step"] = 1e3 * quartets_per_step / out["value"]
        out["extrapolation"] = "whole-step ms = the GPU step's quartet count / the sampled oracle rate"
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2507_09772_gb300 import synth
    import oracle
    mols = synth.batched_631gs(args.nmol)
    sample = oracle_sample(mols, args.oracle_sample)
    for _ in range(args.warmup):
        oracle_pass(sample, args.cutoff)
    nq = 0
    dt = 0.0
    for _ in range(args.steps):
        n, t = oracle_pass(sample, args.cutoff)
        nq += n
        dt += t
    val = nq / dt
    sample_txt = (f"each step: full screened FP64 JK of the {len(sample)} smallest molecules of the batch "
                  f"({min(m.natm for m in sample)}-{max(m.natm for m in sample)} atoms, "
                  f"{nq // max(1, args.steps)} quartets), the sample of the cpu_baseline leg")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "nmol": args.nmol, "precision": "fp64",
                                           "cutoff": args.cutoff,
                                           "sample": f"{len(sample)} smallest molecules"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": sample_txt},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def tier_split(eng, Ds, Js, Ks, args, precision):
    """Class-kernel time per tier of one serialised, per-launch-timed build
    (CUDA events around each launch, one graph branch)."""
    from paper_2507_09772_gb300 import jk
    try:
        eng.set_option("profile", 1)
        eng.set_option("branches", 1)
        _, _, st = eng.build(Ds, cutoff=args.cutoff, precision=precision, J=Js, K=Ks, stats=True)
        ms = {0: 0.0, 1: 0.0}
        q = {0: 0, 1: 0}
        rows = []
        for p in jk.jk_profile(eng.h):
            ms[p["tier"]] += p["ms"]
            q[p["tier"]] += p["quartets"]
            rows.append(dict(p, launches=1))
        out = {"fp64_kernels_ms": ms[0], "fp32_kernels_ms": ms[1], "fp64_quartets": q[0], "fp32_quartets": q[1],
               "serial_build_ms": st["ms"], "timing": "serialised replay, CUDA events around each class launch"}
        probes = {0: getattr(args, "probe64", None), 1: getattr(args, "probe32", None)}
        for t, name in ((0, "fp64_tier_roofline"), (1, "fp32_tier_roofline")):
            out[name] = family_roofline(rows, t, probes[t], st["ms"])
        return out
    except Exception as e:   # a diagnostic, never the reason a run fails
        return {"error": str(e)[:200]}
    finally:
        eng.set_option("profile", 0)
        eng.set_option("branches", args.branches)


def oracle_blocks(mol, nblocks, cutoff, seed=7):
    """Exact J and K shell blocks of one large Cartesian molecule from the CPU
    oracle (row-restricted: J_ab and K_ac straight from eq:jk), half of them
    on nearby shell pairs (the blocks that carry J), half uniform. Returns a
    function that gives max |dJ|, max |dK| of a GPU result on those blocks."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)
    xyz = np.asarray(mol.coords)[mol.shells[:, 0]]

    def pairs(n):
        out = []
        for i in range(n):
            a = int(rng.integers(mol.nshell))
            if i < n // 2:
                near = np.nonzero(np.linalg.norm(xyz - xyz[a], axis=1) < 2.5)[0]
                out.append((a, int(rng.choice(near))))
            else:
                out.append((a, int(rng.integers(mol.nshell))))
        return np.array(out, dtype=np.int64)
    jb, kb = pairs(nblocks), pairs(nblocks)
    t0 = time.perf_counter()
    Jl, Kl, nq = oracle.jk_blocks(mol, jb, kb, cutoff=cutoff)
    secs = time.perf_counter() - t0
    off = np.cumsum([0] + [oracle.ncart(int(l)) for l in mol.shells[:, 1]])

    def compare(J, K):
        J = J.cpu().numpy()[0] if hasattr(J, "cpu") else J[0]
        K = K.cpu().numpy()[0] if hasattr(K, "cpu") else K[0]
        dj = max(float(np.abs(J[off[a]:off[a + 1], off[b]:off[b + 1]] - blk[0]).max()) for (a, b), blk in zip(jb, Jl))
        dk = max(float(np.abs(K[off[a]:off[a + 1], off[c]:off[c + 1]] - blk[0]).max()) for (a, c), blk in zip(kb, Kl))
        return {"max_abs_dJ_oracle": dj, "max_abs_dK_oracle": dk}
    info = {"blocks": f"{nblocks} J and {nblocks} K shell blocks (half on pairs within 2.5 bohr)",
            "oracle_quartets": int(nq), "oracle_s": secs, "cores": oracle.num_threads()}
    return compare, info


def run_forms(args, eng, mols, Ds, Js, Ks, flush, stream, base_ms, base_quartets, ocmp=None):
    """The accelerated forms listed in --forms (mixed: Schwarz x Dmax tiering;
    mixed_asym64: the same with the FP32 tier's large-T Rys limit in FP64;
    mixed_screen32: with the bounds compared in plain FP32; routed: the
    learned router in the band; mixed@<tau32>: another FP32 threshold)
    on the same inputs, timed like the base build (--precision), with their
    largest deviation from the base build over every element of J and K (and,
    for a single large molecule, from the oracle on sampled shell blocks)."""
    import torch
    from paper_2507_09772_gb300 import jk

    base = args.precision
    forms = [f for f in args.forms.split(",") if f and f != base]
    Jref = [j.clone() for j in Js]
    Kref = [k.clone() for k in Ks]
    eng.set_option("tau32", args.tau32)
    out = {base: {"ms_per_step": base_ms, "quartets_per_s": base_quartets / (base_ms * 1e-3)},
           "tau32": args.tau32, "accuracy_reference": f"the {base} build of this run (full matrices)"}

    def timed(precision):
        # the first build of a form compiles (or loads from the disk cache)
        # its kernels and captures its graph: timed on the host, apart
        c0 = eng.get_option("compile_ms")
        t0 = time.perf_counter()
        _, _, st = eng.build(Ds, cutoff=args.cutoff, precision=precision, J=Js, K=Ks, stats=True)  # warm
        torch.cuda.synchronize()
        first_s = time.perf_counter() - t0
        compile_ms = eng.get_option("compile_ms") - c0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        sts = []
        e0.record(stream)
        for _ in range(args.form_steps):
            flush.fill_(1)
            _, _, st = eng.build(Ds, cutoff=args.cutoff, precision=precision, J=Js, K=Ks, stats=True)
            sts.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.form_steps
        dj = max(float((a - b).abs().max()) for a, b in zip(Js, Jref))
        dk = max(float((a - b).abs().max()) for a, b in zip(Ks, Kref))
        st = sts[-1]
        q = st["quartets_fp64"] + st["quartets_fp32"]
        r = {"ms_per_step": ms, "quartets_per_s": q / (ms * 1e-3), f"speedup_vs_{base}": base_ms / ms,
             "max_abs_dJ": dj, "max_abs_dK": dk, "within_1e-8": bool(max(dj, dk) <= 1e-8),
             "fp32_fraction": st["quartets_fp32"] / max(1, q), "quartets_fp64": st["quartets_fp64"],
             "quartets_fp32": st["quartets_fp32"], "quartets_routed": st["quartets_routed"],
             f"same_quartets_as_{base}": bool(q == base_quartets),
             "first_build_s": first_s, "compile_ms": compile_ms}
        if ocmp is not None:
            r.update(ocmp(Js[0], Ks[0]))
        return r

    if "mixed" in forms:
        # the FP32 tier's shapes, tuned on all-FP32 builds (most mixed quartets are FP32)
        t0 = time.perf_counter()
        tune = (eng.autotune(Ds, cutoff=args.cutoff, precision="fp32", max_candidates=3, min_share=0.01)
                if args.tune else None)
        tune_s = time.perf_counter() - t0
        out["mixed"] = timed("mixed")
        out["mixed"]["autotune"] = tune
        out["mixed"]["autotune_s"] = tune_s
        out["mixed"]["tiers"] = tier_split(eng, Ds, Js, Ks, args, "mixed")
    # the mixed build with the large-T Rys limit of the FP32 tier in FP64
    # (asym64 = 1), and with the bounds compared in plain FP32 (screen64 = 0)
    ref_mixed = out["mixed"]["ms_per_step"] if "mixed" in out else (base_ms if base == "mixed" else None)
    for name, opt, val in (("mixed_asym64", "asym64", 1), ("mixed_screen32", "screen64", 0)):
        if name in forms:
            old = eng.get_option(opt)
            eng.set_option(opt, val)
            try:
                out[name] = timed("mixed")
                if ref_mixed:
                    out[name]["cost_vs_mixed"] = out[name]["ms_per_step"] / ref_mixed - 1.0
            finally:
                eng.set_option(opt, old)
    # tau32 calibration: "mixed@<tau32>" times the mixed build at that threshold
    for name in forms:
        if name.startswith("mixed@"):
            tau = float(name.split("@", 1)[1])
            eng.set_option("tau32", tau)
            try:
                out[name] = timed("mixed")
                out[name]["tau32"] = tau
            finally:
                eng.set_option("tau32", args.tau32)
    if "routed" in forms:
        # router: labels from FP64 logging builds of held-out molecules shaped
        # like the batched and cluster workloads (not the ones timed here),
        # trained on the GPU, then routed builds of the workload
        t0 = time.perf_counter()
        from paper_2507_09772_gb300 import synth
        sub = synth.batched_631gs(6, seed_base=5001) + [synth.water_like_cluster(64, seed=5002)]
        eng_l = jk.JK(sub)
        eng_l.set_option("tau32", args.tau32)
        Dl = [torch.tensor(m.D, dtype=torch.float64, device="cuda") for m in sub]
        Jl = [torch.empty_like(d) for d in Dl]
        Kl = [torch.empty_like(d) for d in Dl]
        cap = 2_000_000
        X = torch.empty((cap, 12), dtype=torch.float32, device="cuda")
        y = torch.empty(cap, dtype=torch.float32, device="cuda")
        n = min(cap, jk.jk_router_collect(eng_l.h, Dl, 1, args.cutoff, Jl, Kl, X, y))
        eng_l.close()
        blob, tst = jk.jk_router_train(X[:n], y[:n], steps=1500, batch=8192, lr=2e-3, quantile=0.95, seed=1)
        blob.margin += args.router_margin
        train_s = time.perf_counter() - t0
        eng.load_router(blob)
        r = timed("routed")
        r["tiers"] = tier_split(eng, Ds, Js, Ks, args, "routed")
        r.update({"train_samples": int(n), "train_s": train_s, "margin": float(blob.margin), "train_loss_first": tst["loss_first"],
                  "train_loss_last": tst["loss_last"],
                  "train_set": "FP64 labels of 6 held-out batch molecules and a 64-unit cluster"})
        if ref_mixed:
            r["speedup_vs_mixed"] = ref_mixed / r["ms_per_step"]
        out["routed"] = r
    # leave the base result in Js, Ks
    for a, b in zip(Js, Jref):
        a.copy_(b)
    for a, b in zip(Ks, Kref):
        a.copy_(b)
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_2507_09772_gb300 import dist as jdist
    from paper_2507_09772_gb300 import jk, synth

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    jk.load_library()
    if args.workload == "batch":
        mols = synth.batched_631gs(args.nmol, seed_base=jdist.batch_seed_base(rank))
    elif args.workload == "cluster":
        mols = [synth.water_like_cluster(seed=1002 + 1000 * rank)]
    elif args.workload == "highl":
        mols = [synth.highl_tzvpp(seed=1003 + 1000 * rank)]
    else:
        mols = [synth.router_cluster(seed=1004 + 1000 * rank)]
    t0 = time.perf_counter()
    eng = jk.JK(mols)
    init_s = time.perf_counter() - t0
    eng.set_option("use_graph", args.graph)
    eng.set_option("branches", args.branches)
    if args.chunk:
        eng.set_option("chunk", args.chunk)
    if args.chunk_fp64tier:
        eng.set_option("chunk_fp64tier", args.chunk_fp64tier)
    for kv in args.opt:
        k, v = kv.split("=", 1)
        eng.set_option(k, float(v))
    Ds = [torch.tensor(m.D, dtype=torch.float64, device="cuda") for m in mols]
    Js = [torch.empty_like(d) for d in Ds]
    Ks = [torch.empty_like(d) for d in Ds]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    tune = None
    t0 = time.perf_counter()
    if args.tune:
        tune = eng.autotune(Ds, cutoff=args.cutoff, precision=args.precision, max_candidates=3, min_share=0.01)
    tune_s = time.perf_counter() - t0

    def step(stats=True):
        flush.fill_(1)
        _, _, st = eng.build(Ds, cutoff=args.cutoff, precision=args.precision, J=Js, K=Ks, stats=stats)
        return st

    t0 = time.perf_counter()
    first = step()
    first_s = time.perf_counter() - t0
    first_compile_ms = eng.get_option("compile_ms")
    for _ in range(max(0, args.warmup - 1)):
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e0.record(stream)
    stats = []
    for i in range(args.steps):
        stats.append(step())
        step_ev[i].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    ms_total = e0.elapsed_time(e1)
    step_ms = [(e0 if i == 0 else step_ev[i - 1]).elapsed_time(step_ev[i]) for i in range(args.steps)]

    # Per-kernel launch durations: CUDA events around every class kernel, on
    # the stream it runs on, in steps replayed with the kernels serialised
    # (one graph branch) so that no two class kernels share the GPU.
    eng.set_option("profile", 1)
    eng.set_option("branches", 1)
    prof = {}
    e0.record(stream)
    for _ in range(args.prof_steps):
        step()
        for p in jk.jk_profile(eng.h):
            key = (p["la"], p["lb"], p["lc"], p["ld"], p["na"], p["nb"], p["nc"], p["nd"], p["tier"])
            agg = prof.setdefault(key, dict(p, ms=0.0, flops_model=0.0, quartets=0, launches=0))
            agg["ms"] += p["ms"]
            agg["flops_model"] += p["flops_model"]
            agg["quartets"] += p["quartets"]
            agg["launches"] += 1
    e1.record(stream)
    torch.cuda.synchronize()
    ms_serial = e0.elapsed_time(e1)
    eng.set_option("profile", 0)
    eng.set_option("branches", args.branches)
    quartets = sum(s["quartets_fp64"] + s["quartets_fp32"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    if pg:
        ms_max, q_all = jdist.reduce_step_timing(pg, ms_total, quartets, device="cuda")
    else:
        ms_max, q_all = ms_total, float(quartets)
    value = q_all / (ms_max * 1e-3)

    # roofline of the integral kernel family (FP64 FMA pipe)
    args.probe64 = None if args.no_probe else jk.jk_measure_peak("fp64", 100.0)
    args.probe32 = None if args.no_probe else jk.jk_measure_peak("fp32", 100.0)
    tier = 0 if args.precision == "fp64" else 1
    roofline = family_roofline(list(prof.values()), tier, args.probe64 if tier == 0 else args.probe32,
                               ms_serial / args.prof_steps)
    if args.precision == "mixed":
        roofline["fp64_tier"] = family_roofline(list(prof.values()), 0, args.probe64, ms_serial / args.prof_steps)
    total_kernel_ms = sum(v["ms"] for v in prof.values())
    all_flops = sum(v["flops_model"] for v in prof.values())
    path_fp64 = {"model_tflops": all_flops / (total_kernel_ms * 1e-3) / 1e12,
                 "frac_of_fp64_peak": all_flops / (total_kernel_ms * 1e-3) / PEAK_FP64_NOMINAL}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        Dh = [torch.tensor(m.D, dtype=torch.float64).pin_memory() for m in mols]
        Jh = [torch.empty(d.shape, dtype=torch.float64).pin_memory() for d in Dh]
        Kh = [torch.empty(d.shape, dtype=torch.float64).pin_memory() for d in Dh]
        h2d = sum(d.numel() * 8 for d in Dh)
        d2h = sum(j.numel() * 8 for j in Jh) + sum(k.numel() * 8 for k in Kh)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        e0.record(stream)
        nq = 0
        for _ in range(args.steps):
            flush.fill_(1)
            for d, dh in zip(Ds, Dh):
                d.copy_(dh, non_blocking=True)
            _, _, st = eng.build(Ds, cutoff=args.cutoff, precision=args.precision, J=Js, K=Ks, stats=True)
            nq += st["quartets_fp64"] + st["quartets_fp32"]
            for j, jh in zip(Js, Jh):
                jh.copy_(j, non_blocking=True)
            for k, kh in zip(Ks, Kh):
                kh.copy_(k, non_blocking=True)
            torch.cuda.synchronize()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1)
        if pg:
            t_e, n_e = jdist.reduce_step_timing(pg, ms_e2e, nq, device="cuda")
        else:
            t_e, n_e = ms_e2e, float(nq)
        e2e = {"value": n_e / (t_e * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": t_e / args.steps}

    # a single large Cartesian molecule: sampled oracle blocks for every form
    ocmp, oinfo, fp64_oracle = None, None, None
    if args.oracle_blocks > 0 and len(mols) == 1 and mols[0].natm > 100 and not mols[0].spherical and rank == 0:
        ocmp, oinfo = oracle_blocks(mols[0], args.oracle_blocks, args.cutoff)
        fp64_oracle = ocmp(Js[0], Ks[0])

    # the accelerated forms on the same inputs, against this FP64 build
    forms = None
    if not args.no_forms and args.precision != "fp32":
        forms = run_forms(args, eng, mols, Ds, Js, Ks, flush, stream, ms_max / args.steps, quartets / args.steps,
                          ocmp)
        if fp64_oracle:
            forms[args.precision].update(fp64_oracle)
            forms["oracle_blocks"] = oinfo

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample(mols, args.cpu_seconds, args.cutoff, quartets / args.steps, args.oracle_sample)

    if rank == 0:
        nbf = sum(m.nao for m in mols)
        wl = WORKLOAD if args.workload == "batch" else {
            "cluster": "water-like-cluster-768atm-631gs", "highl": "tzvpp-shaped-60atm-spherical",
            "router": "router-cluster-1024atm-631gs"}[args.workload]
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
            "data": "synthetic",
            "config": {"workload": wl, "nmol": len(mols), "nbf_total": nbf,
                       "natm_range": [min(m.natm for m in mols), max(m.natm for m in mols)],
                       "precision": args.precision, "cutoff": args.cutoff,
                       "l2": "flushed before every step (256 MiB write)",
                       "graph": args.graph, "branches": args.branches,
                       "chunk": eng.get_option("chunk"), "chunk_fp64tier": eng.get_option("chunk_fp64tier"),
                       "screen64": eng.get_option("screen64"), "widen_int": eng.get_option("widen_int"),
                       "options": args.opt,
                       "parallelism": f"{ws} independent batch(es), one per GPU"},
            "quartets_per_step": quartets / args.steps,
            "prim_quartets_per_step": sum(s["prim_quartets"] for s in stats) / args.steps,
            "model_flops_per_step": sum(s["flops_model"] for s in stats) / args.steps,
            "path_fp64_roofline": path_fp64,
            "autotune": tune,
            "serial_ms_per_step": ms_serial / args.prof_steps,
            "step_ms": ({"median": statistics.median(step_ms), "min": min(step_ms), "max": max(step_ms)}
                        if step_ms else None),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "forms": forms,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": int(launches),
            "init_ms": 1e3 * init_s,
            "first_build_s": first_s,
            "compile_ms": first_compile_ms,
            "compile_ms_all_forms": eng.get_option("compile_ms"),
            "autotune_s": tune_s,
            "peak_probe_fp64_tflops": None if args.no_probe else args.probe64 / 1e12,
            "peak_probe_fp32_tflops": None if args.no_probe else args.probe32 / 1e12,
            "top_kernels": sorted(
                [{"class": "(%d%d|%d%d)/%d%d%d%d" % (v["la"], v["lb"], v["lc"], v["ld"], v["na"], v["nb"], v["nc"], v["nd"]),
                  "tier": v["tier"], "ms_per_step": v["ms"] / args.prof_steps, "share": v["ms"] / ms_serial,
                  "quartets_per_step": v["quartets"] / args.prof_steps,
                  "tflops_model": v["flops_model"] / (v["ms"] * 1e-3) / 1e12 if v["ms"] > 0 else 0.0,
                  "G": v["threads_per_quartet"], "regs": v["regs"], "local_bytes": v["local_bytes"]}
                 for v in prof.values()], key=lambda x: -x["ms_per_step"])[:12],
        }
        print(json.dumps(out))
    eng.close()
    if pg:
        pg.destroy_process_group()


def run_micro(args):
    """Micro-benchmarks shaped like the paper's appendix (one JSON line):
    (ss|ss) kernels with n_prim = 1..8 in FP64 and FP32 on a 96-atom cluster
    geometry, and uncontracted d-only / f-only bases on a 192-atom cluster
    geometry with n_dm = 1..4 (time split into a density-independent part and
    a per-density part by a least-squares line in n_dm); then the extended
    forms on 8 molecules of the batched workload (erf / erfc range
    separation, J only, K only, an incremental build of a 1e-8 change) and a
    12-atom uncontracted s p d f g basis (FP64 and mixed)."""
    import numpy as np
    import torch
    from paper_2507_09772_gb300 import jk, synth

    jk.load_library()

    def geometry(nunits, seed):
        rng = np.random.default_rng(seed)
        xyz, _ = synth._triatomic_cluster(rng, nunits)
        return xyz

    def timed_build(eng, D, precision, reps=3):
        eng.build(D, cutoff=args.cutoff, precision=precision, stats=True)   # compile, warm
        ms, st = [], None
        for _ in range(reps):
            _, _, st = eng.build(D, cutoff=args.cutoff, precision=precision, stats=True)
            ms.append(st["ms"])
        return statistics.median(ms), st

    rows = []
    cases = set(args.micro_cases.split(","))
    xyz = geometry(32, 2001)
    for n in (range(1, 9) if "ss" in cases else ()):
        rng = np.random.default_rng(3000 + n)
        exps = np.geomspace(30.0, 0.15, n) if n > 1 else np.array([0.8])
        mol = synth.custom_basis_molecule(xyz, [[(0, exps)] for _ in range(len(xyz))], rng, name=f"s{n}")
        eng = jk.JK(mol)
        D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
        m64, s64 = timed_build(eng, D, "fp64")
        m32, s32 = timed_build(eng, D, "fp32")
        eng.close()
        rows.append({"case": "(ss|ss)", "natm": len(xyz), "n_prim": n, "ms_fp64": m64, "ms_fp32": m32,
                     "fp64_over_fp32": m64 / m32, "quartets": s64["quartets_fp64"],
                     "prim_quartets": s64["prim_quartets"]})
    xyz = geometry(args.micro_units, 2002)
    for l, name in ((2, "d-only"), (3, "f-only")):
        if name[0] not in cases:
            continue
        rng = np.random.default_rng(4000 + l)
        per_atom = [[(l, np.array([np.exp(rng.uniform(np.log(0.4), np.log(1.2)))]))] for _ in range(len(xyz))]
        mol = synth.custom_basis_molecule(xyz, per_atom, rng, n_dm=4, name=name)
        eng = jk.JK(mol)
        pts = []
        for ndm in range(1, 5):
            D = torch.tensor(mol.D[:ndm], dtype=torch.float64, device="cuda")
            ms, st = timed_build(eng, D, "fp64")
            pts.append((ndm, ms))
            rows.append({"case": name, "natm": len(xyz), "nao": mol.nao, "n_dm": ndm, "ms_fp64": ms,
                         "quartets": st["quartets_fp64"]})
        eng.close()
        a = np.polyfit([p[0] for p in pts], [p[1] for p in pts], 1)
        rows.append({"case": name, "fit": "ms = integrals + n_dm * per_density",
                     "integrals_ms": float(a[1]), "per_density_ms": float(a[0])})
    if "forms" not in cases:
        print(json.dumps({"micro": rows, "cutoff": args.cutoff, "data": "synthetic"}))
        return
    # the "next" forms on 8 molecules of the batched workload: range
    # separation, J-only / K-only, and an incremental build of a small change
    mols = synth.batched_631gs(8)
    eng = jk.JK(mols)
    Ds = [torch.tensor(m.D, dtype=torch.float64, device="cuda") for m in mols]
    for name, opts, kw in (("coulomb", {}, {}), ("erf w=0.3", {"omega": 0.3}, {}),
                           ("erfc w=0.3", {"omega": -0.3}, {}), ("J only", {}, {"with_k": False}),
                           ("K only", {}, {"with_j": False})):
        try:
            for k, v in opts.items():
                eng.set_option(k, v)
            eng.build(Ds, cutoff=args.cutoff, stats=True, **kw)
            ms = []
            for _ in range(3):
                _, _, st = eng.build(Ds, cutoff=args.cutoff, stats=True, **kw)
                ms.append(st["ms"])
            rows.append({"case": "batch8 " + name, "ms_fp64": statistics.median(ms),
                         "quartets": st["quartets_fp64"]})
        except Exception as e:
            rows.append({"case": "batch8 " + name, "error": str(e)[:200]})
        finally:
            eng.set_option("omega", 0.0)
    try:
        rng = np.random.default_rng(9)
        dD = [torch.tensor(1e-8 * (lambda x: x + x.T)(rng.standard_normal(m.D.shape[1:]))[None],
                           dtype=torch.float64, device="cuda") for m in mols]
        eng.build(dD, cutoff=args.cutoff, stats=True)
        ms = []
        for _ in range(3):
            _, _, st = eng.build(dD, cutoff=args.cutoff, stats=True)
            ms.append(st["ms"])
        rows.append({"case": "batch8 incremental |dD| ~ 1e-8", "ms_fp64": statistics.median(ms),
                     "quartets": st["quartets_fp64"]})
    except Exception as e:
        rows.append({"case": "batch8 incremental", "error": str(e)[:200]})
    eng.close()
    # g shells: 12 atoms, uncontracted s p d f g on each
    try:
        rng = np.random.default_rng(4004)
        xyz = geometry(4, 2003)
        per_atom = [[(l, np.array([np.exp(rng.uniform(np.log(0.3), np.log(2.0)))])) for l in range(5)]
                    for _ in range(len(xyz))]
        mol = synth.custom_basis_molecule(xyz, per_atom, rng, name="spdfg")
        eng = jk.JK(mol)
        D = torch.tensor(mol.D, dtype=torch.float64, device="cuda")
        m64, s64 = timed_build(eng, D, "fp64")
        m32, _ = timed_build(eng, D, "mixed")
        eng.close()
        rows.append({"case": "spdfg uncontracted", "natm": len(xyz), "nao": mol.nao, "ms_fp64": m64,
                     "ms_mixed": m32, "quartets": s64["quartets_fp64"]})
    except Exception as e:
        rows.append({"case": "spdfg uncontracted", "error": str(e)[:200]})
    print(json.dumps({"micro": rows, "cutoff": args.cutoff, "data": "synthetic"}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.micro:
        run_micro(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark of the damage-weighted TLSPH step: pair-interactions per second.

Workload (default): the Johnson-Cook tensile bar, a 40x40x640 jittered simple
cubic lattice (1,024,000 particles, about 1.0e8 directed neighbour pairs) at
0.5 mm spacing, cubic spline h = 1.5 spacing, neighbours within 2h, grips at
+-1 m/s, dt = 0.3 CFL.  Synthetic, seeded inputs.

A pair-interaction is one directed pair (i, j in S_i) advanced through one
full step (both gather passes).  `value` is device-timed with CUDA events on
the stream the library launches on, inputs resident in HBM; `e2e` is the same
metric through the C ABI with host buffers: upload of the specimen from
pinned memory, neighbour build, the K steps (each followed by a read-back of
its diagnostics: momentum, force sum, kinetic and internal energy, failures) and the
download of the final fields, all inside the timed region.  The state a step reads and writes
(about 0.9 GB of HBM traffic) is far larger than the 129 MB L2, so no flush is
needed between steps.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded
prefix of the same bar (same metric and unit).
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

METRIC = "pair-interactions/s (mixed vs FP64 GPU, same accuracy); served p50/p99 latency"
UNIT = "pair-interactions/s"


# ---------------------------------------------------------------- workloads
def workload(name: str):
    from paper_1901_07374_gb300 import specimen as S
    if name == "tensile_bar_jc_40x40x640":
        return S.tensile_bar_jc()
    if name == "tensile_bar_jc_40x40x160":
        return S.tensile_bar_jc(nz=160)
    if name == "tensile_bar_cl_8x8x32":
        return S.tensile_bar_cl()
    if name == "notched_bar_gtn":
        return S.notched_bar_gtn()
    if name == "taylor_impact_500k":
        return S.taylor_impact(500000, v_impact=200.0)
    raise SystemExit(f"unknown workload {name}")


# bars pulled along z by grips at both ends: their plastic-flow window starts
# from an affine stretch (specimen.plastic_flow_state)
GRIPPED_BARS = ("tensile_bar", "notched_bar")


def algorithmic_bytes(N: int, nnz: int, precision: str, list_words: int | None = None) -> dict:
    """Bytes each pass must move between HBM and the SMs per step: the
    neighbour lists (the CSR column index of every pair, or the mixed path's
    sliced lists: `list_words` 4-byte words) plus every particle's own state
    read and written once (gathered neighbour data counts as on-chip reuse).
    Per-pass per-particle figures follow the state layout of the library."""
    if precision == "fp64":
        p1 = 4 * nnz + 656 * N     # row_ptr 8, X 24, v 24, Linv 72, F rw 144, sd rw 96, scalars rw 64,
        #                            D r+w 16, fail 4, mat 4, sigma r+w 96, e r+w 16, A w 72, vol 16 (gathered only)
        p2 = 4 * nnz + 357 * N     # row_ptr 8, X 24, u 24, F 72, A 72, D 8, vol 8, E 8, mass 8,
        #                            vh rw 48, v w 24, force w 24, u' w 24, fail 4, bc 1
    else:
        from paper_1901_07374_gb300 import tlsph
        p1, p2 = tlsph.mixed_algorithmic_bytes(N, nnz if list_words is None else list_words)
    return {"pass1": p1, "pass2": p2}


# DRAM bytes (read + write) per launch of each pass from one ncu capture
# (profiles/traffic_tensile_bar_jc_40x40x640.md), keyed by (workload,
# precision, pass, plan form of that pass) and stamped with the digest of the
# CUDA sources they were captured from: a figure is reported only while the
# sources are unchanged (otherwise `traffic` is null until the next capture).
TRAFFIC_SOURCES = "e6cc72b91479d63571156f6acb48bdfce3161c74b68082d8707498a63375bcbc"
TRAFFIC = {
    ("tensile_bar_jc_40x40x640", "mixed", "pass1", 4): 597210624,    # k_gather1_mixed_t4 + k_epi1_mixed + k_epi1_slow
    ("tensile_bar_jc_40x40x640", "mixed", "pass1", 5): 1098680832,   # k_gather1_mixed_t4w (weight table) + the same
    ("tensile_bar_jc_40x40x640", "mixed", "pass2", 7): 327032320,    # k_pass2_mixed_tc5
    ("tensile_bar_jc_40x40x640", "mixed", "pass2", 8): 327364864,    # k_pass2_mixed_tc5p
}


def kernel_sources_digest() -> str:
    """SHA-256 over the code of the library's CUDA sources and headers (sorted
    by name; comments and whitespace left out, so editing a comment keeps the
    stamp while any change to the code drops it)."""
    import glob
    import hashlib
    import re
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_1901_07374_gb300", "csrc", "*.cu*"))
                    + [os.path.join(ROOT, "include", "tlsph.h")]):
        with open(p, encoding="utf-8") as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(os.path.basename(p).encode())
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()


def profiled_traffic(workload: str, precision: str, kern: str, form: int):
    """DRAM bytes of one launch from the ncu capture of the current sources, or None."""
    if TRAFFIC_SOURCES is None or TRAFFIC_SOURCES != kernel_sources_digest():
        return None
    return TRAFFIC.get((workload, precision, kern, form))


def max_over_ranks(value: float, dist, device=None) -> float:
    """The largest value over all ranks (a timing: the job ends with its
    slowest rank); identity on one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(seconds: float, max_steps: int | None = None, nz: int = 24, warmup: int = 1):
    """Pair-interactions/s of the FP64 oracle (single thread) on the first
    `nz` layers of the 40x40 bar; `warmup` untimed steps, then stepping until
    `seconds` or max_steps.  Returns (rate, steps, pairs per step, N, seconds)."""
    import oracle
    from paper_1901_07374_gb300 import specimen as S
    w = S.tensile_bar_jc(nx=40, ny=40, nz=nz)
    sim = oracle.Simulation.from_workload(w)
    sim.step(max(1, warmup))
    steps = 0
    t0 = time.perf_counter()
    while True:
        sim.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_steps and steps >= max_steps):
            break
    return sim.nnz * steps / el, steps, sim.nnz, sim.N, el


def _oracle_replica(seconds: float, q) -> None:
    q.put(oracle_rate(seconds)[0])


def oracle_rate_all_cores(seconds: float, cores: int | None = None):
    """Aggregate pair-interactions/s of `cores` independent single-thread
    oracle replicas (spawned processes, one per host core) stepping the same
    bounded sample side by side: the host's all-core oracle throughput.  The
    oracle sums each row sequentially, so every replica computes the same
    bits as the single-thread run."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_replica, args=(seconds, q)) for _ in range(cores)]
    for p in procs:
        p.start()
    rates = [q.get() for _ in procs]
    for p in procs:
        p.join()
    return sum(rates), cores


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    warmup = max(1, args.warmup)
    rate, steps, nnz, N, el = oracle_rate(1e9, max_steps=args.steps, warmup=warmup)
    sample = f"first 24 of 640 layers of the 40x40 bar ({N} particles, {nnz} pairs), {steps} steps in {el:.1f} s"
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample": sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
FIELDS = ("U", "V", "F", "SIGMA", "STRESS_DEV", "EPSP", "DINIT", "DAMAGE", "FORCE")


def field_scales(w) -> dict:
    """Floor of the normwise relative error of each field: spacing, grip
    speed, yield stress, yield stress x spacing^2, 1e-3 for strains/damage."""
    import numpy as np
    sp = w.specimen
    L = sp.spacing
    v = float(np.abs(sp.bc_vel).max()) or 1.0
    s = max(w.materials[0]["A"], 1e6)
    return dict(U=L, V=v, F=1.0, SIGMA=s, STRESS_DEV=s, EPSP=1e-3, DINIT=1e-3, DAMAGE=1e-3, FORCE=s * L * L)


def launches_per_step(plan) -> int:
    """Kernels one step launches: FP64 path 2; mixed plans 1 or 2 per pass plus
    the FP64-update kernel of pass 1."""
    if not plan:
        return 2
    return (2 if plan[0] >= 2 else 1) + 1 + (2 if plan[2] == 2 else 1)


def field_errors(sim, ref: dict, sc: dict) -> dict:
    """Normwise relative error of each field of `sim` against the state dict
    `ref` (floors `sc`), and the size of the symmetric difference of the
    failure sets."""
    import numpy as np
    out = {}
    for f in FIELDS:
        a, b = sim.get(f), ref[f]
        out[f] = float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), sc[f]))
    out["failure_set_symdiff"] = int(((sim.get("FAIL_STEP") >= 0) ^ (ref["FAIL_STEP"] >= 0)).sum())
    return out


def plastic_errors(a, b, sc: dict) -> dict:
    """Field errors of `a` against `b` (normwise relative max with the floors
    `sc`, and RMS), the number of particles whose plastic strain differs by
    more than 1e-8, and the size of the symmetric difference of the failure
    sets."""
    import numpy as np
    out = {}
    for f in FIELDS:
        x, y = a.get(f), b.get(f)
        out[f] = float(np.max(np.abs(x - y)) / max(float(np.max(np.abs(y))), sc[f]))
        out[f + "_rms"] = float(np.sqrt(np.mean((x - y) ** 2)) / max(float(np.sqrt(np.mean(y ** 2))), sc[f]))
    d = np.abs(a.get("EPSP") - b.get("EPSP"))
    out["particles_epsp_diff_above_1e-8"] = int((d > 1e-8).sum())
    out["failure_set_symdiff"] = int(((a.get("FAIL_STEP") >= 0) ^ (b.get("FAIL_STEP") >= 0)).sum())
    return out


def timed_run(tlsph, torch, w, precision, steps, warmup, stream, clocks=None, plan=None, state=None, guard=None,
              prestep=0):
    """Create, warm up, then time `steps` steps with CUDA events on the
    library's stream; per-kernel times from the library's own events.  A
    mixed context takes `plan`, else the autotuner's; `state` (caller-order
    fields) is loaded before the warm-up."""
    sim = tlsph.Simulation.from_workload(w, precision=precision, stream=stream)
    N, nnz, _ = sim.info()
    words = None
    if precision == "mixed":
        from paper_1901_07374_gb300 import autotune
        if plan:
            sim.set_plan(plan)
        else:
            autotune.tune(sim)
        pl, lw = sim.get_plan(), sim.neighbor_layout()["words"]
        words = (lw if pl[0] in (1, 2, 4) else nnz, lw if pl[2] != 0 else nnz)
        if guard is not None:
            sim.set_guard(guard)
    for k, v in (state or {}).items():
        sim.set(k, v)
    if prestep:
        sim.step(prestep)       # untimed: move the run to the window of interest (e.g. after an impact)
    sim.step(warmup)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    sim.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    p1, p2, nprof = sim.profile_read()
    sim.profile(False)
    clk = clocks.stop() if clocks else None
    sim.sync()
    return sim, dict(ms=ms, p1=p1 / max(1, nprof), p2=p2 / max(1, nprof), N=N, nnz=nnz, clocks=clk,
                     plan=sim.get_plan() if precision == "mixed" else None, words=words,
                     layout=sim.neighbor_layout() if precision == "mixed" else None)


def run_ours(args, rank: int, world: int, dist):
    import ctypes

    import numpy as np
    import torch

    from paper_1901_07374_gb300 import tlsph

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = workload(args.workload)
    sp = w.specimen
    stream = torch.cuda.current_stream()
    if dist:
        dist.barrier()

    # ---- FP64 GPU path (the comparison) and the headline precision
    ref_sim, ref = (None, None)
    if args.precision != "fp64" and not args.skip_fp64:
        ref_sim, ref = timed_run(tlsph, torch, w, "fp64", args.steps, args.warmup, stream, prestep=args.prestep)
    sim, r = timed_run(tlsph, torch, w, args.precision, args.steps, args.warmup, stream,
                       clocks=ClockSampler(torch.cuda.current_device()), plan=args.plan, prestep=args.prestep)
    N, nnz, ms = r["N"], r["nnz"], r["ms"]
    ms = max_over_ranks(ms, dist, "cuda")
    value = world * nnz * args.steps / (ms * 1e-3)

    # ---- accuracy of the headline path against the FP64 GPU path (same steps)
    accuracy = None
    ref_state = None
    if ref_sim is not None:
        sc = field_scales(w)
        ref_state = {f: ref_sim.get(f) for f in FIELDS + ("FAIL_STEP",)}
        accuracy = field_errors(sim, ref_state, sc)
        accuracy["steps"] = args.prestep + args.warmup + args.steps
        ref_sim.close()
    sim.close()

    # ---- guard band of the FP32 elastic screen: throughput and accuracy per band
    guard = None
    if args.guard_sweep and args.precision == "mixed" and ref_state is not None:
        from paper_1901_07374_gb300 import specimen as S
        st = S.plastic_flow_state(w) if args.workload.startswith(GRIPPED_BARS) else None
        guard = []
        for band in (1e-5, 1e-3, 1e-1, 1.0):
            gs, gr = timed_run(tlsph, torch, w, "mixed", args.steps, args.warmup, stream, plan=r.get("plan"),
                               guard=band)
            row = {"band": band, "ms_per_step": gr["ms"] / args.steps,
                   "max_error_vs_fp64": max(v for k, v in field_errors(gs, ref_state, field_scales(w)).items()
                                            if k != "failure_set_symdiff")}
            gs.close()
            if st is not None:
                ps, pr = timed_run(tlsph, torch, w, "mixed", args.plastic_steps, args.warmup, stream,
                                   plan=r.get("plan"), state=st, guard=band)
                row["plastic_ms_per_step"] = pr["ms"] / args.plastic_steps
                ps.close()
            guard.append(row)

    # ---- roofline of the dominant kernel: HBM bytes and FP32 issue
    words = r.get("words") or (nnz, nnz)
    ab = {"pass1": algorithmic_bytes(N, nnz, args.precision, words[0])["pass1"],
          "pass2": algorithmic_bytes(N, nnz, args.precision, words[1])["pass2"]}
    kern = "pass2" if r["p2"] >= r["p1"] else "pass1"
    k_ms = r[{"pass1": "p1", "pass2": "p2"}[kern]]
    peaks = measured_peaks()
    peak, src = peaks.get("hbm_gbs"), "measured"
    if not peak:
        peak, src = 6800.0, "fallback"
    achieved = ab[kern] / (k_ms * 1e-3) / 1e9
    hbm = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_source": src,
           "traffic": profiled_traffic(args.workload, args.precision, kern,
                                       (r.get("plan") or (0, 0, 0, 0))[0 if kern == "pass1" else 2]),
           "algorithmic_bytes_per_launch": ab[kern]}
    roofline = hbm
    if args.precision == "mixed":
        ops = dict(zip(("pass1", "pass2"), tlsph.mixed_fp32_ops(nnz, w.hg_alpha != 0.0)))
        peak_alu = tlsph.FP32_LANES * 2070e6 / 1e12
        ach_alu = ops[kern] / (k_ms * 1e-3) / 1e12
        try:
            fma32 = tlsph.fma_peak(False, 4096) / 1e12
            fma64 = tlsph.fma_peak(True, 128) / 1e12
        except tlsph.TlsphError:
            fma32 = fma64 = None
        roofline = {"bound": "alu", "kernel": kern, "achieved": ach_alu, "peak": peak_alu, "unit": "TFLOP/s",
                    "frac": ach_alu / peak_alu,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz (an FMA counts as one op)",
                    "measured_fma_peak": {"fp32": fma32, "fp64": fma64, "unit": "T FMA/s"},
                    "frac_of_measured_fp32": ach_alu / fma32 if fma32 else None,
                    "traffic": hbm["traffic"], "algorithmic_ops_per_launch": ops[kern],
                    "fp32_ops_per_pair": tlsph.MIXED_FP32_OPS_PER_PAIR, "hbm_view": hbm}
    roofline["ms_per_launch"] = {"pass1": r["p1"], "pass2": r["p2"]}

    # ---- the same bar with every particle in plastic flow (FP64 return in both paths)
    plastic = None
    if not args.no_plastic and args.workload.startswith(GRIPPED_BARS):
        from paper_1901_07374_gb300 import specimen as S
        st = S.plastic_flow_state(w)
        ps, pr = timed_run(tlsph, torch, w, args.precision, args.plastic_steps, args.warmup, stream,
                           plan=r.get("plan"), state=st)
        plastic = {"steps": args.plastic_steps, "ms_per_step": pr["ms"] / args.plastic_steps,
                   "value": world * nnz * args.plastic_steps / (pr["ms"] * 1e-3),
                   "ms_per_launch": {"pass1": pr["p1"], "pass2": pr["p2"]},
                   "plastic_fraction": float(np.mean(ps.get("EPSP") > 0))}
        if args.precision != "fp64" and not args.skip_fp64:
            qs, qr = timed_run(tlsph, torch, w, "fp64", args.plastic_steps, args.warmup, stream, state=st)
            plastic["fp64_value"] = world * nnz * args.plastic_steps / (qr["ms"] * 1e-3)
            sc = field_scales(w)
            plastic["accuracy_vs_fp64"] = plastic_errors(ps, qs, sc)
            if args.rate_free_control:
                # control: the same window without the rate term of Eq. JC_viscoplastic_model (C = 0)
                import dataclasses
                m0 = dict(w.materials[0])
                m0["C"] = 0.0
                w0 = dataclasses.replace(w, materials=[m0] + list(w.materials[1:]))
                cs_, _ = timed_run(tlsph, torch, w0, "mixed", args.plastic_steps, args.warmup, stream,
                                   plan=r.get("plan"), state=st)
                cq_, _ = timed_run(tlsph, torch, w0, "fp64", args.plastic_steps, args.warmup, stream, state=st)
                plastic["rate_free_control"] = {"C": 0.0, "accuracy_vs_fp64": plastic_errors(cs_, cq_, sc)}
                cs_.close()
                cq_.close()
            qs.close()
        ps.close()

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        def pinned(a):
            t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            return t, t.numpy()
        keep = [pinned(a) for a in (sp.X, sp.vol, sp.mat_id, sp.bc_mask, sp.bc_vel, sp.f0)]
        X, vol, mat, bcm, bcv, f0 = (k[1] for k in keep)
        outs = {k: pinned(np.empty((N, c))) for k, c in (("U", 3), ("V", 3), ("SIGMA", 9), ("DAMAGE", 1))}
        h2d = sum(k[1].nbytes for k in keep)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        s2 = tlsph.Simulation(X, vol, mat, bcm, bcv, f0, w.materials, w.h, w.rc, w.dt, w.hg_alpha,
                              precision=args.precision, stream=stream)
        if r.get("plan"):
            s2.set_plan(r["plan"])
        d2h = 0
        diag = None
        # each step's result read back: the step's diagnostics, copied into page-locked buffers behind the
        # step and read by the host while the next step runs (two buffers, an event each)
        bufs = [torch.empty(tlsph.DIAG_COUNT, dtype=torch.float64).pin_memory() for _ in range(2)]
        evs = [torch.cuda.Event() for _ in range(2)]
        for k in range(args.steps):
            s2.step(1)
            s2.diagnostics_async(bufs[k % 2])
            evs[k % 2].record(stream)
            d2h += tlsph.DIAG_COUNT * 8
            if k > 0:
                evs[(k - 1) % 2].synchronize()
                diag = tlsph.diagnostics_dict(bufs[(k - 1) % 2])
        if args.steps > 0:
            evs[(args.steps - 1) % 2].synchronize()
            diag = tlsph.diagnostics_dict(bufs[(args.steps - 1) % 2])
        L = tlsph.load()
        for k, (t, a) in outs.items():
            tlsph._check(L.tlsph_get_state(s2.ctx, tlsph.FIELD[k], a.ctypes.data_as(ctypes.c_void_p), a.nbytes, 0),
                         s2.ctx)
            d2h += a.nbytes
        el = time.perf_counter() - t0
        s2.close()
        el = max_over_ranks(el, dist, "cuda")
        e2e = {"value": world * nnz * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "includes": "create (upload of the specimen from pinned memory, neighbour build, L^-1) + the tuned "
                           "plan + K steps, each followed by a read-back of its diagnostics (momentum, force sum, "
                           "kinetic and internal energy, failures) into page-locked memory, read by the host while "
                           "the next step runs + download of u, v, sigma, D",
               "final_kinetic_energy": diag["kinetic_energy"] if diag else None}

    # ---- the metric's batched and served forms, small versions inside the default run
    batched = served = None
    if args.precision == "mixed" and not args.no_forms:
        from paper_1901_07374_gb300 import specimen as S
        batched = measure_batched(tlsph, torch, S.batched_specimens(args.forms_specimens, seed=0), args.steps,
                                  args.warmup, stream, fp64_one_by_one=True)
        batched["workload"] = (f"the first {args.forms_specimens} bars of the 256-bar batched workload "
                               "(same generator and seed)")
        summ = serve_once(args, args.rate, count=args.forms_requests, steps_range=(200, 1000))
        served = {"workload": f"{args.forms_requests} requests of the serving stream (same generator and seed, "
                              f"Poisson arrivals at {args.rate:g}/s, half Taylor cylinders and half bars) with "
                              "200-1000 steps each instead of 1000-5000, 120 GB admission cap",
                  "latency_s": {"p50": summ["p50_s"], "p95": summ["p95_s"], "p99": summ["p99_s"]},
                  "pair_interactions_per_s": summ["pair_interactions_per_s"],
                  "offered_pair_interactions_per_s": summ["offered_pair_interactions_per_s"],
                  "makespan_s": summ["makespan_s"], "done": summ["done"], "failed": summ["failed"],
                  "max_live": summ["max_live"], "peak_mem_gb": summ["peak_mem_gb"], "steps": summ["steps"],
                  "clocks": summ["clocks"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, steps, onnz, oN, oel = oracle_rate(args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first 24 of 640 layers of the bar ({oN} particles, {onnz} pairs), "
                         f"{steps} steps in {oel:.1f} s, single thread"}
        if args.cpu_all_cores:
            agg, cores = oracle_rate_all_cores(args.cpu_seconds / 2)
            cpu["replicas_on_all_cores"] = {"value": agg, "unit": UNIT, "cores": cores,
                                            "how": "independent single-thread oracle replicas of the same sample, "
                                                   "one per host core (the oracle itself is single-threaded)"}
    if rank != 0:
        return
    cfg = {"workload": args.workload, "precision": args.precision, "particles": N, "pairs_per_step": nnz,
           "prestep": args.prestep,
           "particle_steps_per_s": world * N * args.steps / (ms * 1e-3),
           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
           "l2": "inputs larger than L2 (about 0.9 GB of HBM traffic per step vs 129 MB)"}
    if r.get("layout"):
        cfg["neighbor_lists"] = dict(r["layout"], bytes_per_pair=4.0 * r["layout"]["words"] / nnz)
    if plastic:
        cfg["plastic_flow_window"] = plastic
    if guard:
        cfg["guard_sweep"] = guard
    if batched:
        cfg["batched"] = batched
    if served:
        cfg["served"] = served
    if ref is not None:
        cfg["plan"] = r.get("plan")
        cfg["fp64_gpu_value"] = world * nnz * args.steps / (ref["ms"] * 1e-3)
        cfg["fp64_ms_per_launch"] = {"pass1": ref["p1"], "pass2": ref["p2"]}
        cfg["accuracy_vs_fp64"] = accuracy
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic (seeded jittered lattice)", "config": cfg,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step(r.get("plan")) * args.steps,
            "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batched and served forms
# ---------------------------------------------------------------- accuracy trajectories
ACCURACY_CHECKPOINTS = (1, 10, 100, 500, 2000)


def accuracy_cases():
    """Workloads of the mixed-vs-FP64 trajectory report: the two
    failure-exercising 8x8x32 bars (Cockcroft-Latham and Johnson-Cook damage),
    the 1.02M-particle Johnson-Cook bar as specified, and the GTN notched bar."""
    from paper_1901_07374_gb300 import specimen as S
    return {
        "tensile_bar_cl_8x8x32_failure": lambda: S.failure_variant(S.tensile_bar_cl(steps=2000)),
        "tensile_bar_jc_8x8x32_failure": lambda: S.failure_variant(S.tensile_bar_jc(nx=8, ny=8, nz=32, steps=2000)),
        "tensile_bar_jc_40x40x640": lambda: S.tensile_bar_jc(),
        "notched_bar_gtn": lambda: S.notched_bar_gtn(steps=2000),
    }


def trajectory_errors(a, b, sc: dict) -> dict:
    """Max and RMS normwise relative error of every field of `a` (mixed)
    against `b` (FP64), the symmetric difference of the failure sets and the
    distribution of the failure-step differences of particles failed in both."""
    import numpy as np
    out = {}
    fa, fb = a.get("FAIL_STEP"), b.get("FAIL_STEP")
    live = (fa < 0) & (fb < 0)
    for f in FIELDS:
        x, y = a.get(f), b.get(f)
        out[f] = {"max": float(np.max(np.abs(x - y)) / max(float(np.max(np.abs(y))), sc[f])),
                  "rms": float(np.sqrt(np.mean((x - y) ** 2)) / max(float(np.sqrt(np.mean(y ** 2))), sc[f]))}
        if not live.all() and live.any():   # the particles that have not failed in either path
            xl, yl = x[live], y[live]
            out[f]["max_live"] = float(np.max(np.abs(xl - yl)) / max(float(np.max(np.abs(yl))), sc[f]))
    both = (fa >= 0) & (fb >= 0)
    d = (fa[both] - fb[both]).astype(np.int64)
    out["failed"] = {"fp64": int((fb >= 0).sum()), "mixed": int((fa >= 0).sum()),
                     "symdiff": int(((fa >= 0) ^ (fb >= 0)).sum())}
    out["fail_step_delta"] = ({"n": int(d.size), "nonzero": int((d != 0).sum()), "min": int(d.min()),
                               "max": int(d.max()), "mean_abs": float(np.abs(d).mean())} if d.size else {"n": 0})
    return out


def run_accuracy(args):
    """Mixed against the FP64 GPU path along whole trajectories, reported at
    fixed step counts (not gated: the tests gate the FP64 path against the
    oracle and the mixed path over short windows).  One JSON line per
    workload."""
    from paper_1901_07374_gb300 import tlsph
    cases = accuracy_cases()
    names = args.accuracy_cases.split(",") if args.accuracy_cases else list(cases)
    for name in names:
        w = cases[name]()
        sc = field_scales(w)
        a = tlsph.Simulation.from_workload(w, precision="mixed")
        b = tlsph.Simulation.from_workload(w, precision="fp64")
        N, nnz, _ = b.info()
        rows, done, t0 = {}, 0, time.perf_counter()
        for k in ACCURACY_CHECKPOINTS:
            a.step(k - done)
            b.step(k - done)
            done = k
            rows[str(k)] = trajectory_errors(a, b, sc)
        print(json.dumps({"accuracy": name, "particles": N, "pairs": nnz, "checkpoints": rows,
                          "seconds": time.perf_counter() - t0}), flush=True)
        a.close()
        b.close()


def measure_batched(tlsph, torch, ws, steps: int, warmup: int, stream, fp64_one_by_one: bool = False) -> dict:
    """Advance the specimens `ws` together (one persistent launch per kernel
    kind and step, replayed from a CUDA graph) and, for comparison, the same
    mixed contexts stepped one by one and (optionally) FP64 contexts of the
    same specimens stepped one by one.  Device-timed with CUDA events."""
    t0 = time.perf_counter()
    sims = [tlsph.Simulation.from_workload(w, precision="mixed", stream=stream, line_order=True) for w in ws]
    setup = time.perf_counter() - t0
    N = sum(s.N for s in sims)
    nnz = sum(s.nnz for s in sims)
    lays = [s.neighbor_layout() for s in sims]
    b = tlsph.Batch(len(sims), stream=stream)
    b.set(sims)
    from paper_1901_07374_gb300 import autotune
    t1 = time.perf_counter()
    shape = autotune.tune_batch(b, sims)            # launch shapes of the batch kernels (state restored)
    tune_s = time.perf_counter() - t1
    b.step(warmup)
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    # the same contexts, each with its own launches, one after another per step
    for s in sims:
        s.sync()
    e0.record(stream)
    for _ in range(steps):
        for s in sims:
            s.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    for s in sims:
        s.sync()
    b.close()
    for s in sims:
        s.close()
    out = {"specimens": len(ws), "particles": N, "pairs_per_step": nnz, "set_up_s": setup,
           "ms_per_step": ms / steps, "value": nnz * steps / (ms * 1e-3),
           "one_by_one_value": nnz * steps / (ms_seq * 1e-3), "one_by_one_ms_per_step": ms_seq / steps,
           "kernel_launches_per_step": {"batched": 5, "one_by_one": 4 * len(ws)},
           "list_words": sum(x["words"] for x in lays), "launch_shape": list(shape), "tune_s": tune_s,
           "clocks": clocks}
    if fp64_one_by_one:
        f64 = [tlsph.Simulation.from_workload(w, precision="fp64", stream=stream) for w in ws]
        for s in f64:
            s.step(1)
        torch.cuda.synchronize()
        k = max(1, steps // 4)
        e0.record(stream)
        for _ in range(k):
            for s in f64:
                s.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        out["fp64_one_by_one_value"] = nnz * k / (e0.elapsed_time(e1) * 1e-3)
        out["fp64_steps_timed"] = k
        for s in f64:
            s.close()
    return out


def run_batched(args):
    """256 independent bars (log-uniform 2k..200k particles, JC constants
    +-20%) advanced together: one persistent launch per kernel kind and step
    replayed from a CUDA graph, against the same contexts stepped one by one."""
    import torch

    from paper_1901_07374_gb300 import specimen as S
    from paper_1901_07374_gb300 import tlsph
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    ws = S.batched_specimens(args.specimens, seed=0)
    stream = torch.cuda.current_stream()
    m = measure_batched(tlsph, torch, ws, args.steps, args.warmup, stream)
    N, nnz, ms = m["particles"], m["pairs_per_step"], m["ms_per_step"] * args.steps
    p1, p2 = algorithmic_bytes(N, nnz, "mixed", m["list_words"]).values()
    achieved = (p1 + p2) / (ms / args.steps * 1e-3) / 1e9
    peak = measured_peaks().get("hbm_gbs") or 6800.0
    ops = sum(tlsph.mixed_fp32_ops(nnz, True))       # every member with hourglass control
    peak_alu = tlsph.FP32_LANES * 2070e6 / 1e12
    ach_alu = ops / (ms / args.steps * 1e-3) / 1e12
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded jittered lattices)",
            "config": {"workload": f"batched_{len(ws)}", "specimens": len(ws), "particles": N,
                       "pairs_per_step": nnz, "set_up_s": m["set_up_s"],
                       "one_by_one_value": m["one_by_one_value"],
                       "one_by_one_ms_per_step": m["one_by_one_ms_per_step"],
                       "kernel_launches_per_step": m["kernel_launches_per_step"],
                       "launch_shape": m["launch_shape"]},
            "roofline": {"bound": "alu", "kernel": "whole step (five launches)", "achieved": ach_alu,
                         "peak": peak_alu, "unit": "TFLOP/s", "frac": ach_alu / peak_alu,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz (an FMA counts as one op)",
                         "traffic": None, "algorithmic_ops_per_step": ops,
                         "hbm_view": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                      "frac": achieved / peak, "traffic": None}},
            "gpu_launches": 5 * args.steps, "clocks": m["clocks"]}
    print(json.dumps(line), flush=True)


def serve_once(args, rate, count=None, steps_range=(1000, 5000)):
    import torch

    from paper_1901_07374_gb300 import serve
    from paper_1901_07374_gb300 import specimen as S
    stream_reqs = S.serving_requests(count=count or args.requests, rate=rate, seed=0, steps_range=steps_range)
    reqs = [serve.Request(k, t, w, n) for k, (t, w, n) in enumerate(stream_reqs)]
    srv = serve.Server(mem_cap_bytes=120e9, chunk_steps=args.chunk)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    t0 = time.perf_counter()
    srv.run(reqs, realtime=True)
    makespan = time.perf_counter() - t0
    clocks = clk.stop()
    summ = serve.summarize(reqs, makespan)
    offered = rate * sum(r.pairs * r.steps for r in reqs) / max(1, len(reqs))
    summ.update(rate_per_s=rate, offered_pair_interactions_per_s=offered, peak_mem_gb=srv.peak_used / 1e9,
                max_live=max((n for _, n, _ in srv.timeline), default=0),
                steps=int(sum(r.steps for r in reqs)), clocks=clocks)
    return summ


def run_serving(args):
    """Poisson stream of tensile bars and Taylor-impact cylinders, 1000-5000
    steps each, served by continuous batching under a 120 GB device-memory
    cap: the configured rate (20/s) and, with --rates, a sweep of arrival rates
    on the same request seeds (latency knee)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rates = sorted({float(x) for x in args.rates.split(",")} | {args.rate}) if args.rates else [args.rate]
    runs = {rate: serve_once(args, rate) for rate in rates}
    head = runs[args.rate]
    sweep = None
    if len(rates) > 1:
        base = runs[rates[0]]["p99_s"]
        knee = next((r for r in rates if runs[r]["p99_s"] > 2.0 * base), None)
        sweep = {"knee_rate_per_s": knee,
                 "knee_definition": "lowest arrival rate whose p99 latency exceeds twice the p99 at the lowest rate",
                 "runs": [{k: runs[r][k] for k in ("rate_per_s", "p50_s", "p95_s", "p99_s", "makespan_s",
                                                  "pair_interactions_per_s", "offered_pair_interactions_per_s",
                                                  "done", "max_live", "peak_mem_gb")} for r in rates]}
    line = {"metric": METRIC, "value": head["pair_interactions_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": head["steps"], "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic request stream",
            "config": {"workload": "serving", "requests": args.requests, "rate_per_s": args.rate,
                       "chunk_steps": args.chunk, "mem_cap_gb": 120, "peak_mem_gb": head["peak_mem_gb"],
                       "latency_s": {"p50": head["p50_s"], "p95": head["p95_s"], "p99": head["p99_s"]},
                       "makespan_s": head["makespan_s"], "done": head["done"], "failed": head["failed"],
                       "max_live": head["max_live"], "rate_sweep": sweep},
            "clocks": head["clocks"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default=None)
    ap.add_argument("--workload", default="tensile_bar_jc_40x40x640")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--accuracy", action="store_true",
                    help="report mixed vs FP64 along whole trajectories (steps 1, 10, 100, 500, 2000) and exit")
    ap.add_argument("--accuracy-cases", default="", help="comma-separated subset of the accuracy workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", dest="cpu_all_cores", action="store_false",
                    help="skip the all-core oracle figure (one replica per host core)")
    ap.add_argument("--skip-fp64", action="store_true", help="do not run the FP64 comparison path")
    ap.add_argument("--specimens", type=int, default=256, help="batched workload: number of specimens")
    ap.add_argument("--requests", type=int, default=32, help="serving workload: number of requests")
    ap.add_argument("--rate", type=float, default=20.0, help="serving workload: arrivals per second")
    ap.add_argument("--chunk", type=int, default=100, help="serving workload: steps per batch chunk")
    ap.add_argument("--rates", default=None, help="serving workload: comma-separated arrival-rate sweep")
    ap.add_argument("--plan", default=None, help="mixed launch plan v1,b1,v2,b2 (default: autotuned)")
    ap.add_argument("--no-plastic", action="store_true", help="skip the plastic-flow window")
    ap.add_argument("--plastic-steps", type=int, default=10)
    ap.add_argument("--prestep", type=int, default=0, help="untimed steps before the warm-up (both paths)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and served records of the default run")
    ap.add_argument("--forms-specimens", type=int, default=32, help="default run: bars in the batched record")
    ap.add_argument("--forms-requests", type=int, default=16, help="default run: requests in the served record")
    ap.add_argument("--rate-free-control", action="store_true",
                    help="plastic-flow window: also compare the paths with the Johnson-Cook rate term off (C = 0)")
    ap.add_argument("--guard-sweep", action="store_true",
                    help="time the mixed path at several guard bands of its FP32 elastic screen")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.plan:
        args.plan = tuple(int(x) for x in args.plan.split(","))
    if args.precision is None:
        from paper_1901_07374_gb300 import tlsph
        args.precision = tlsph.DEFAULT_PRECISION
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.accuracy:
        run_accuracy(args)
        return
    if args.workload.startswith("batched"):
        run_batched(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    run_ours(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

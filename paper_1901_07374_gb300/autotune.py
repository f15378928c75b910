"""Launch-plan autotuner of the mixed-precision step.

A plan is (pass-1 form, pass-1 block, pass-2 form, pass-2 block); every plan
computes the same method (see tlsph_set_plan).  The tuner times each
candidate of a pass with the library's own CUDA events on the context's
stream, keeps the fastest per pass, and restores the simulation state
bit for bit afterwards (checkpoint of every resumable field, step counter
included), so tuning never changes a trajectory.  Results are cached per
(GPU, precision, particle-count bucket, neighbours-per-row bucket, hourglass
on/off, candidate set) in a JSON file ($TLSPH_PLAN_CACHE, default
~/.cache/tlsph_gb300/plans.json).

Batches (tlsph.Batch) are tuned the same way: `tune_batch` chooses the
launch-shape variant of each batch kernel kind (register cap and pairs in
flight of the pass-1 gather, the per-particle update and pass 2) by timing
whole batched steps one kind at a time, and restores every member's state
bit for bit.
"""
from __future__ import annotations

import json
import math
import os
import threading
import zlib

from .tlsph import TlsphError

PASS1 = [(0, 128), (1, 128), (2, 64), (2, 128), (2, 256), (3, 256), (4, 64), (4, 128), (4, 256), (5, 64), (5, 128)]
PASS2 = [(0, 128), (1, 64), (1, 128), (1, 256), (2, 128), (3, 128), (3, 256), (4, 64), (4, 128), (5, 128), (6, 64),
         (6, 128), (7, 64), (7, 128), (8, 128)]
DEFAULT = (4, 64, 4, 128)

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("TLSPH_PLAN_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "tlsph_gb300",
                                                              "plans.json")


def _key(sim) -> str:
    import torch
    N, nnz, _ = sim.info()
    name = torch.cuda.get_device_name()
    hg = "hg" if sim.cfg.hg_alpha != 0 else "nohg"
    # the candidate lists are part of the key: a cached plan is only reused by a tuner that would choose among
    # the same candidates
    cand = zlib.crc32(repr((PASS1, PASS2, DEFAULT)).encode())
    return (f"{name}|{sim.precision}|N2^{int(math.log2(max(N, 1)))}|row{int(round(nnz / max(N, 1) / 8.0)) * 8}|{hg}"
            f"|c{cand:08x}")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, plan) -> None:
    path = cache_path()
    with _lock:
        d = _load()
        d[key] = list(plan)
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(d, f, indent=1, sort_keys=True)
            os.replace(tmp, path)
        except OSError:
            pass


def _time(sim, plan, steps: int, warmup: int):
    sim.set_plan(plan)
    sim.step(warmup)
    sim.profile(True)
    sim.step(steps)
    p1, p2, n = sim.profile_read()
    sim.profile(False)
    return p1 / max(n, 1), p2 / max(n, 1)


def tune(sim, steps: int = 3, warmup: int = 1, use_cache: bool = True, record=None):
    """Choose and set the fastest plan for `sim` (a mixed-precision
    tlsph.Simulation); returns it.  `record`, if a list, receives
    (plan, ms pass 1, ms pass 2) for every timed candidate."""
    if sim.precision != "mixed":
        return None
    key = _key(sim)
    if use_cache:
        cached = _load().get(key)
        if cached:
            sim.set_plan(cached)
            return tuple(cached)
    ck = sim.checkpoint(device=True)
    plan0 = sim.get_plan()
    best1, best2 = None, None
    for v1, b1 in PASS1:
        plan = (v1, b1, DEFAULT[2], DEFAULT[3])
        try:
            t1, t2 = _time(sim, plan, steps, warmup)
        except TlsphError:
            if v1 != 5:         # pass-1 form 5 needs library-owned memory for its weight table
                raise
            continue
        if record is not None:
            record.append((plan, t1, t2))
        if best1 is None or t1 < best1[0]:
            best1 = (t1, v1, b1)
    for v2, b2 in PASS2:
        plan = (best1[1], best1[2], v2, b2)
        t1, t2 = _time(sim, plan, steps, warmup)
        if record is not None:
            record.append((plan, t1, t2))
        if best2 is None or t2 < best2[0]:
            best2 = (t2, v2, b2)
    sim.restore(ck)
    best = (best1[1], best1[2], best2[1], best2[2])
    sim.set_plan(best if best else plan0)
    if use_cache:
        _store(key, best)
    return best


def _batch_key(batch, sims) -> str:
    import torch
    N = sum(s.N for s in sims)
    nnz = sum(s.nnz for s in sims)
    hg = "hg" if sims and sims[0].cfg.hg_alpha != 0 else "nohg"
    _, nv = batch.get_shape()
    return (f"batch|{torch.cuda.get_device_name()}|N2^{int(math.log2(max(N, 1)))}"
            f"|m2^{int(math.log2(max(len(sims), 1)))}|row{int(round(nnz / max(N, 1) / 8.0)) * 8}|{hg}|v{nv}")


def _time_batch(batch, shape, steps: int, warmup: int) -> float:
    import torch
    batch.set_shape(shape)
    batch.step(warmup, graph=True)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.step(steps, graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune_batch(batch, sims, steps: int = 3, warmup: int = 1, use_cache: bool = True, record=None):
    """Choose and set the fastest launch shape for `batch` (whose members are
    the Simulations `sims`); returns it.  Coordinate descent: each kernel
    kind's variants are timed (whole graph-replayed steps, CUDA events on the
    current stream) with the other kinds at their best so far.  Every member's
    resumable state and step counter are restored bit for bit afterwards, so
    tuning never changes a trajectory.  `record`, if a list, receives
    (shape, ms per step) for every timed candidate."""
    key = _batch_key(batch, sims)
    if use_cache:
        cached = _load().get(key)
        if cached:
            batch.set_shape(cached)
            return tuple(cached)
    cks = [s.checkpoint(device=True) for s in sims]
    best, nv = batch.get_shape()
    best = list(best)
    for kind in range(3):
        times = {}
        for v in range(nv[kind]):
            shape = list(best)
            shape[kind] = v
            t = _time_batch(batch, shape, steps, warmup)
            times[v] = t
            if record is not None:
                record.append((tuple(shape), t))
        best[kind] = min(times, key=times.get)
    for s, ck in zip(sims, cks):
        s.restore(ck)
    batch.set(sims)
    batch.set_shape(best)
    if use_cache:
        _store(key, best)
    return tuple(best)

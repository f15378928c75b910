"""Continuous-batching server for TLSPH simulation requests.

A request is a specimen (workload) and a number of steps.  The server keeps
every admitted request's state resident on the GPU and advances all live
requests together through one tlsph batch (one persistent launch per kernel
kind and step, replayed from a CUDA graph).  Between chunks of steps it

* admits requests that have arrived, first come first served, while the
  device-memory estimate of the live set stays under the cap; a newly
  admitted request is created on its own stream while the batch's steps of
  the others are still running, so set-up overlaps with the stepping;
* retires requests whose steps are done: their final fields are copied to
  the host and their device memory is released;
* cancels requests on demand.

Chunks end exactly where the next live request finishes (at most
`chunk_steps` long), so no request takes more steps than it asked for.  A
request's result does not depend on which others shared its batch (the batch
kernels compute each context independently).

Latency is completion time minus arrival time; throughput is the total
pair-interactions of all requests over the makespan.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import tlsph

# neighbours per particle allowed for in the memory estimate: 122 is the
# most a +-1% jittered cubic lattice can have within 3 spacings
NBR_BOUND = 122


@dataclasses.dataclass
class Request:
    id: int
    arrival: float              # seconds after the start of the run
    workload: object            # specimen.Workload
    steps: int
    admitted: float = None
    done: float = None
    status: str = "pending"     # pending | live | done | failed | cancelled
    error: str = None
    result: dict = None
    pairs: int = 0

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


def memory_estimate(w, precision: str = "mixed") -> int:
    """Device bytes a request needs: the context workspace for the bound on
    neighbours plus its sliced-ELL copy."""
    N = w.specimen.N
    cfg = tlsph.make_config(w.h, w.rc, w.dt, w.hg_alpha, precision)
    nnz = N * NBR_BOUND
    ws = tlsph.workspace_bytes(cfg, N, nnz)
    return int(ws + (nnz + nnz // 2) * 4 if precision == "mixed" else ws)


class Server:
    def __init__(self, mem_cap_bytes: float = 120e9, max_live: int = 512, chunk_steps: int = 100,
                 precision: str = "mixed", graph: bool = True, fields=("U", "V", "SIGMA", "DAMAGE", "FAIL_STEP"),
                 clock=time.perf_counter, line_order: bool = True):
        import torch
        self.cap = int(mem_cap_bytes)
        self.max_live = int(max_live)
        self.chunk = int(chunk_steps)
        self.precision = precision
        self.graph = graph
        self.fields = tuple(fields)
        # lattice-line internal order: the many small specimens of a request mix carry far fewer padding slots
        self.line_order = line_order
        self.clock = clock
        self.create_stream = torch.cuda.Stream()
        self.batch = tlsph.Batch(self.max_live, stream=torch.cuda.current_stream())
        self.live = []              # [request, simulation, steps left, bytes]
        self.used = 0
        self.peak_used = 0
        self.cancel_ids = set()
        self.timeline = []          # (time, live count, bytes in use)

    # ---------------------------------------------------------------- helpers
    def _admit(self, r: Request, now: float) -> bool:
        need = memory_estimate(r.workload, self.precision)
        if need > self.cap:
            r.status, r.error, r.done = "failed", f"needs {need} bytes, over the cap", now
            return True
        if self.used + need > self.cap or len(self.live) >= self.max_live:
            return False
        try:
            sim = tlsph.Simulation.from_workload(r.workload, precision=self.precision, stream=self.create_stream,
                                                 line_order=self.line_order and self.precision == "mixed")
        except (tlsph.TlsphError, RuntimeError, ValueError) as e:
            r.status, r.error, r.done = "failed", str(e), now
            return True
        r.status, r.admitted = "live", now
        r.pairs = sim.nnz
        self.live.append([r, sim, r.steps, need])
        self.used += need
        self.peak_used = max(self.peak_used, self.used)
        return True

    def _retire(self, entry, now: float, status: str):
        r, sim, _, need = entry
        if status == "done":
            r.result = {k: sim.get(k) for k in self.fields}
        r.status, r.done = status, now
        sim.close()
        self.used -= need

    def cancel(self, request_id: int) -> None:
        """Cancel a pending or live request (takes effect at the next chunk)."""
        self.cancel_ids.add(request_id)

    # ---------------------------------------------------------------- main loop
    def run(self, requests, realtime: bool = True):
        """Serve `requests` (list of Request, any order).  With realtime the
        arrivals follow the wall clock; otherwise a request counts as arrived
        as soon as the server asks.  Returns the requests with their times,
        status and results."""
        import torch
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock()
        members_dirty = True
        while pending or self.live:
            now = self.clock() - t0
            # cancellations
            for e in [e for e in self.live if e[0].id in self.cancel_ids]:
                self.live.remove(e)
                self._retire(e, now, "cancelled")
                members_dirty = True
            for r in [r for r in pending if r.id in self.cancel_ids]:
                pending.remove(r)
                r.status, r.done = "cancelled", now
            # admission, first come first served
            while pending and (pending[0].arrival <= now or not realtime):
                if not self._admit(pending[0], now):
                    break
                pending.pop(0)
                members_dirty = True
            if not self.live:
                if pending and realtime:
                    time.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            if members_dirty:
                self.create_stream.synchronize()
                self.batch.set([e[1] for e in self.live])
                members_dirty = False
            k = min(self.chunk, min(e[2] for e in self.live))
            self.batch.step(k, graph=self.graph)
            # while the GPU steps the live set, set up requests that arrived meanwhile
            now = self.clock() - t0
            while pending and (pending[0].arrival <= now or not realtime) and pending[0].id not in self.cancel_ids:
                if not self._admit(pending[0], now):
                    break
                pending.pop(0)
                members_dirty = True
            self.batch.sync()
            torch.cuda.current_stream().synchronize()
            now = self.clock() - t0
            for e in list(self.live):
                e[2] -= k
                if e[2] == 0:
                    self.live.remove(e)
                    self._retire(e, now, "done")
                    members_dirty = True
            self.timeline.append((now, len(self.live), self.used))
        return requests


def summarize(requests, makespan: float) -> dict:
    """Latency percentiles (seconds) and throughput of a finished run."""
    done = [r for r in requests if r.status == "done"]
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    pair_steps = float(sum(r.pairs * r.steps for r in done))
    return {"requests": len(requests), "done": len(done),
            "failed": sum(r.status == "failed" for r in requests),
            "cancelled": sum(r.status == "cancelled" for r in requests),
            "p50_s": float(np.percentile(lat, 50)), "p95_s": float(np.percentile(lat, 95)),
            "p99_s": float(np.percentile(lat, 99)), "makespan_s": makespan,
            "pair_interactions_per_s": pair_steps / makespan if makespan > 0 else 0.0}

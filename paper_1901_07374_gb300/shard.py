"""Specimen-level sharding with halo exchange (one rank per GPU, host side).

Rows (particles) are split into slabs along the specimen's longest axis with
balanced particle counts.  A rank owns its slab's rows and keeps, as halo,
every particle outside its slab that is a neighbour of one of its rows.  The
neighbour sets are fixed in the reference configuration (Sec. 2.2), so the
halo lists and the exchange schedule are built once.

Local numbering keeps the global order (owned and halo particles sorted by
global index), so the neighbours of an owned row appear in the same order as
on one device and every sum over j runs in the same order: a sharded run
reproduces the single-domain result bit for bit.

A step has two exchange points (velocity-Verlet step of the method):
  after the predictor  the halo needs v^{n+1/2}, u^{n+1} and D^n, which the
                       pass-1 gather reads (Sec. 3.1, Fdot);
  after pass 1         the halo needs A, D^{n+1}, F and u^{n+1}, which the
                       pass-2 gather reads (Sec. 3.1 forces, hourglass term).
At each point a rank sends to each neighbouring rank the rows of its own
particles that lie in that rank's halo, and receives its halo rows from their
owners (point-to-point over torch.distributed: NCCL between GPUs, gloo on
CPU).  Halo rows are recomputed locally by the backend in between, but every
value a neighbour reads is the owner's, so their partial neighbourhoods never
leak into an owned row.

The stepping backend is anything with predict / pass1 / pass2 phases and
per-particle state arrays over the local particles; the tests drive the FP64
oracle this way on CPU ranks.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def partition_slabs(X: np.ndarray, nranks: int) -> np.ndarray:
    """Owner rank of every particle: contiguous slabs along the longest
    bounding-box axis holding N / nranks particles each (ties in the
    coordinate broken by particle index)."""
    X = np.asarray(X, np.float64)
    N = X.shape[0]
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    axis = int(np.argmax(X.max(axis=0) - X.min(axis=0))) if N else 0
    order = np.lexsort((np.arange(N), X[:, axis]))
    owner = np.empty(N, np.int32)
    owner[order] = (np.arange(N, dtype=np.int64) * nranks // max(N, 1)).astype(np.int32)
    return owner


def halo_of(row_ptr: np.ndarray, col: np.ndarray, owner: np.ndarray, rank: int) -> np.ndarray:
    """Global indices (ascending) of the particles outside `rank`'s slab that
    are neighbours of its rows."""
    rows = np.nonzero(owner == rank)[0]
    if rows.size == 0:
        return np.zeros(0, np.int64)
    starts, ends = row_ptr[rows], row_ptr[rows + 1]
    need = np.concatenate([col[a:b] for a, b in zip(starts, ends)]) if rows.size else np.zeros(0, np.int64)
    need = np.unique(need.astype(np.int64))
    return need[owner[need] != rank]


@dataclasses.dataclass
class HaloPlan:
    """One rank's share of a sharded specimen.

    local:      global indices of the local particles (owned and halo), ascending
    owned:      (len(local),) bool, True for the rank's own rows
    row_ptr, col: the local neighbour CSR (local indices; rows of halo
                particles keep only their local neighbours)
    send[s]:    local indices of own particles in rank s's halo (ascending global index)
    recv[s]:    local indices of halo particles owned by rank s (ascending global index)
    """

    rank: int
    nranks: int
    local: np.ndarray
    owned: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray
    send: dict
    recv: dict

    @classmethod
    def build(cls, row_ptr, col, owner, rank: int) -> "HaloPlan":
        row_ptr = np.asarray(row_ptr, np.int64)
        col = np.asarray(col, np.int64)
        owner = np.asarray(owner, np.int32)
        nranks = int(owner.max()) + 1 if owner.size else 1
        mine = np.nonzero(owner == rank)[0]
        halo = halo_of(row_ptr, col, owner, rank)
        local = np.union1d(mine, halo)
        g2l = np.full(owner.shape[0], -1, np.int64)
        g2l[local] = np.arange(local.size)
        owned = owner[local] == rank
        # local CSR: each local row keeps its neighbours that are local, in global (= local) order
        lrp = np.zeros(local.size + 1, np.int64)
        parts = []
        for k, g in enumerate(local):
            nb = g2l[col[row_ptr[g]:row_ptr[g + 1]]]
            nb = nb[nb >= 0]
            parts.append(nb)
            lrp[k + 1] = lrp[k] + nb.size
        lcol = np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
        send, recv = {}, {}
        for s in range(nranks):
            if s == rank:
                continue
            hs = halo_of(row_ptr, col, owner, s)                 # rank s's halo
            out = hs[owner[hs] == rank]                           # ... that this rank owns
            inc = halo[owner[halo] == s]                          # this rank's halo owned by s
            if out.size:
                send[s] = g2l[out]
            if inc.size:
                recv[s] = g2l[inc]
        return cls(rank, nranks, local, owned, lrp, lcol, send, recv)

    def peers(self) -> list:
        return sorted(set(self.send) | set(self.recv))


def exchange(plan: HaloPlan, arrays: dict, group=None) -> None:
    """Overwrite every halo row of each array (first axis = local particle)
    with its owner's row.  Rows travel as one contiguous buffer per array and
    peer; sends are posted first, then receives, so no ordering deadlock."""
    import torch
    import torch.distributed as dist
    pending, unpack = [], []
    for name in sorted(arrays):
        a = arrays[name]
        for s in plan.peers():
            if s in plan.send:
                buf = torch.from_numpy(np.ascontiguousarray(a[plan.send[s]]))
                pending.append(dist.isend(buf, dst=s, group=group))
                unpack.append(None)
        for s in plan.peers():
            if s in plan.recv:
                idx = plan.recv[s]
                buf = torch.empty((idx.size,) + a.shape[1:], dtype=torch.from_numpy(a[:0]).dtype)
                pending.append(dist.irecv(buf, src=s, group=group))
                unpack.append((a, idx, buf))
    for req, up in zip(pending, unpack):
        req.wait()
        if up is not None:
            a, idx, buf = up
            a[idx] = buf.numpy()


class ShardedStepper:
    """Drives a backend through sharded steps: predict, exchange, pass 1,
    exchange, pass 2.  The backend provides predict(), pass1(), pass2() over
    its local particles and state() -> dict of the per-particle arrays that
    neighbours read (views that the exchange overwrites in place)."""

    def __init__(self, plan: HaloPlan, backend, group=None):
        self.plan = plan
        self.backend = backend
        self.group = group

    def step(self, n: int = 1) -> None:
        b = self.backend
        for _ in range(n):
            b.predict()
            exchange(self.plan, b.state(), self.group)
            b.pass1()
            exchange(self.plan, b.state(), self.group)
            b.pass2()

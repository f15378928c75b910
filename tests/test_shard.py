"""Specimen-level sharding with halo exchange, on CPU ranks (gloo).

The plan (slabs, halo lists, exchange schedule) is checked for its invariants;
then 2 and 3 ranks step their slabs of a failure-exercising bar with the FP64
oracle as the backend, exchanging halo rows after the predictor and after
pass 1, and the owned rows must equal the single-domain oracle run bit for bit
(local numbering keeps the global order of every sum over j)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1901_07374_gb300 import shard
from paper_1901_07374_gb300 import specimen as S

FIELDS = ("u", "v", "F", "sd", "sigma", "A", "ep", "epdot", "dinit", "D", "f", "force")


def workload():
    return S.failure_variant(S.tensile_bar_cl(nx=5, ny=5, nz=30, steps=40))


def test_partition_and_halo_plan_invariants():
    w = workload()
    X = w.specimen.X
    row_ptr, col = oracle.neighbors(X, w.rc)
    N = X.shape[0]
    for nranks in (1, 2, 3, 4):
        owner = shard.partition_slabs(X, nranks)
        counts = np.bincount(owner, minlength=nranks)
        assert counts.sum() == N and counts.max() - counts.min() <= 1
        plans = [shard.HaloPlan.build(row_ptr, col, owner, r) for r in range(nranks)]
        for p in plans:
            g = p.local
            assert np.all(np.diff(g) > 0)
            assert np.array_equal(np.sort(g[p.owned]), np.nonzero(owner == p.rank)[0])
            # every owned row keeps all its neighbours, in the global order
            for k in np.nonzero(p.owned)[0]:
                gi = g[k]
                assert np.array_equal(g[p.col[p.row_ptr[k]:p.row_ptr[k + 1]]], col[row_ptr[gi]:row_ptr[gi + 1]])
            # what s receives from r is exactly what r sends to s
            for s, idx in p.recv.items():
                q = plans[s]
                assert np.array_equal(g[idx], q.local[q.send[p.rank]])
                assert np.all(owner[g[idx]] == s) and not np.any(p.owned[idx])
        if nranks == 1:
            assert not plans[0].send and not plans[0].recv


class OracleBackend:
    """The FP64 oracle over one rank's local particles (owned + halo)."""

    def __init__(self, w, plan):
        sp = w.specimen
        i = plan.local
        self.sim = oracle.Simulation(sp.X[i], sp.vol[i], sp.mat_id[i], sp.bc_mask[i], sp.bc_vel[i], sp.f0[i],
                                     w.materials, w.h, w.rc, w.dt, w.hg_alpha,
                                     neighbors_csr=(plan.row_ptr, plan.col), wall=w.wall)

    def predict(self):
        self.sim.step_phase("predict")

    def pass1(self):
        self.sim.step_phase("pass1")

    def pass2(self):
        self.sim.step_phase("pass2")

    def state(self):
        d = {k: self.sim[k] for k in FIELDS}
        d["vh"] = self.sim.vh
        d["fail_step"] = self.sim.fail_step
        return d


def _rank_main(rank, world, port, steps, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = workload()
        row_ptr, col = oracle.neighbors(w.specimen.X, w.rc)
        owner = shard.partition_slabs(w.specimen.X, world)
        plan = shard.HaloPlan.build(row_ptr, col, owner, rank)
        be = OracleBackend(w, plan)
        shard.ShardedStepper(plan, be).step(steps)
        own = plan.owned
        res = {k: v[own] for k, v in be.state().items()}
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), ids=plan.local[own], **res)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_oracle_matches_single_domain_bitwise(world, tmp_path):
    import torch.multiprocessing as mp
    steps = 40
    w = workload()
    ref = oracle.Simulation.from_workload(w)
    ref.step(steps)
    mp.start_processes(_rank_main, args=(world, _free_port(), steps, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    seen = np.zeros(w.specimen.N, bool)
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        ids = d["ids"]
        assert not seen[ids].any()
        seen[ids] = True
        for k in FIELDS:
            assert np.array_equal(d[k], ref[k][ids]), (r, k)
        assert np.array_equal(d["fail_step"], ref.fail_step[ids])
        assert np.array_equal(d["vh"], ref.vh[ids])
    assert seen.all()
    assert (ref.fail_step >= 0).any() or (ref["ep"] > 0).any()

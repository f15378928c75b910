"""The benchmark's multi-rank logic on CPU ranks (gloo, world size 2).

Each rank times a different amount of work; the job time every rank reports
is the slowest rank's (max over ranks), and the whole-job throughput counts
the units of all ranks.  Under the reference arm only rank 0 runs and prints;
the other ranks return without work."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = 1.5 + 2.0 * rank                     # rank r's own elapsed time
        job = bench.max_over_ranks(mine, dist)
        dist.barrier()
        buf = io.StringIO()

        class A:
            steps = 1
            workload = "tensile_bar_jc_40x40x640"
        if rank != 0:                              # rank 0 would time the oracle for minutes
            with redirect_stdout(buf):
                bench.run_reference(A, rank, world)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"job": job, "printed": buf.getvalue()}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, None) == 3.25


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_reference_rank_rule_on_gloo(world, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    slowest = 1.5 + 2.0 * (world - 1)
    assert all(r["job"] == slowest for r in res)
    assert all(r["printed"] == "" for r in res[1:])

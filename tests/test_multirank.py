"""The N > 1 path of bench.py on CPU with two gloo ranks (the path shards as independent
replicas, so there is no data-path collective to test): every rank gets its own seeds,
the timing is the maximum over ranks, and the job value is all ranks' particle updates
over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        seeds = {name: [r["seed"] for r in bench.rows_of(name, rank)] for name in ("scan48", "cfg2", "cfg5")}
        my_s = 1.0 + rank  # this rank's "time"
        t_max = bench.max_over_ranks_of(my_s, world, "cpu")
        upd = bench.particle_updates(bench.rows_of("cfg2", rank), 1000, 0, 10)
        out[rank] = (seeds, t_max, bench.job_value(world, upd, t_max), upd)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    (s0, t0, v0, u0), (s1, t1, v1, u1) = out[0], out[1]
    for name in s0:  # every replica of a workload draws its own particles
        assert not set(s0[name]) & set(s1[name]), name
    assert t0 == t1 == 2.0  # the slowest rank's time on every rank
    assert u0 == u1 == 10 * 1000
    assert v0 == v1 == pytest.approx(2 * 10 * 1000 / 2.0)

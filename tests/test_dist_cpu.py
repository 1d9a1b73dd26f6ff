"""The multi-GPU path is replicas only: every rank solves its own bodies and the
ranks exchange nothing but the job-level timing and counts.  Checked here
with two gloo ranks on the CPU: the body shards are disjoint and cover the job,
and the job figures are the slowest rank's time and the sum of solved units."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, bodies, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.body_seeds(rank, bodies)
    ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    solved = 32 * len(seeds) - rank     # rank 1 missed one RHS
    t, n = bench.aggregate_over_ranks(ms, solved, "cpu")
    out[rank] = (tuple(seeds), t, n)
    dist.destroy_process_group()


def test_replica_sharding_and_job_aggregate_gloo():
    world, bodies = 2, 3
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, bodies, out), nprocs=world, join=True)
        res = dict(out)
    s0, s1 = set(res[0][0]), set(res[1][0])
    assert not (s0 & s1) and len(s0 | s1) == world * bodies
    for r in range(world):
        assert res[r][1] == pytest.approx(150.0)      # max over ranks
        assert res[r][2] == 2 * 32 * bodies - 1       # sum over ranks

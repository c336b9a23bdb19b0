"""The multi-GPU form is replicas only: each rank runs independent seeded
starts and the benchmark reduces only its timing (max over ranks).  These
tests run that host logic on 2 CPU ranks over gloo."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import qf_inputs as qi

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is slower
    mx = bench.max_over_ranks(ms, dist, "cpu")
    inst = qi.make_problem(3, qi.brickwork_locations(3, 2), 2, seed=bench.replica_seed(rank))
    out[rank] = (mx, float(inst.starts.real.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_distinct_replicas():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 15.0  # both ranks see the slowest rank's time
    assert out[0][1] != out[1][1]  # replicas draw different starts


def test_job_throughput_counts_every_rank():
    import bench

    # 1056 updates per rank per step, 2 ranks, 10 steps in 500 ms
    assert bench.job_throughput(1056, 2, 10, 500.0) == pytest.approx(1056 * 2 * 10 / 0.5)

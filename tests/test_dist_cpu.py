"""The N > 1 path of bench.py on CPU: two gloo ranks, each its own replica.

The run shards by trajectory (replicas, weak scaling); the only collective is
the max of the timing over ranks.  Checked here without a GPU: the max and the
job rate over two ranks, distinct replica seeds, and the reference arm
returning at once on every rank but 0.
"""
import os
import socket
import sys

import pytest
import torch.distributed as tdist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [2.0, 3.5][rank]                       # rank 1 is the slower replica
        slowest = bench.max_over_ranks(seconds, tdist, "cpu")
        out[rank] = (slowest, bench.job_rate(10, world, slowest), bench.replica_seed(rank))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_replicas():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 3.5
    assert out[0][1] == out[1][1] == pytest.approx(20 / 3.5)
    assert out[0][2] != out[1][2]


def test_single_process_needs_no_group_and_reference_arm_skips_other_ranks():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, None, "cpu") == 1.25
    assert bench.job_rate(4, 1, 2.0) == 2.0

    class A:
        natoms = 8
    assert bench.run_reference(A(), 2, 1) == 0        # rank 1 of 2 does no work

"""The replicas-only multi-GPU path of bench.py, on CPU: two gloo ranks.

Instances are independent, so N GPUs run N replicas of the batch with no
collective on the data path; the only cross-rank steps are the barrier before
the timed region and the max-over-ranks of the timed milliseconds, from which
the whole-job rate is formed.  Those two steps run here with world size 2 on
the gloo backend (127.0.0.1 rendezvous), without a GPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        tdist.barrier()
        ms_local = [12.5, 40.0][rank]            # the second replica is the slow one
        ms = bench.max_over_ranks(ms_local)      # CPU tensor under gloo
        rate = bench.whole_job_rate(1968 * 10, ms, world)
        out[rank] = (ms, rate)
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1]
    ms, rate = out[0]
    assert ms == 40.0
    assert rate == pytest.approx(2 * 1968 * 10 / 0.040)


def test_single_process_is_a_no_op():
    import bench
    assert bench.max_over_ranks(7.25) == 7.25
    assert bench.whole_job_rate(100, 10.0, 1) == pytest.approx(1e4)

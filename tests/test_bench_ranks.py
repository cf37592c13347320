"""The multi-GPU path of bench.py runs N independent replicas (the method has
no exchange step): replicas are timed by the slowest rank and the job's
ms/frame is that time over N.  Checked here with two gloo ranks on the CPU;
the reference arm does no work on ranks other than 0."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [30.0, 50.0][rank]                      # this rank's timed ms
        slow = bench.reduce_max(local, world)
        dist.barrier()
        out[rank] = (slow, bench.job_ms_per_frame(slow / 5, world))
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0] == out[1] == (50.0, 5.0)             # max over ranks, 5 steps, 2 replicas


def test_single_process_helpers():
    import bench
    assert bench.reduce_max(12.5, 1) == 12.5
    assert bench.job_ms_per_frame(12.0, 1) == 12.0
    assert bench.job_ms_per_frame(12.0, 4) == 3.0


def test_reference_arm_idles_on_other_ranks():
    import bench
    assert bench.run_reference(None, 1, 2) is None      # rank 1 of 2 returns before any work

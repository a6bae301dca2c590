"""The N > 1 host logic of bench.py on the CPU: two gloo ranks (world size 2,
127.0.0.1) run the same max-over-ranks reduction the GPU ranks run over NCCL,
and the whole-job value counts every rank's bytes over the slowest rank's
time.  The path has no exchange step (replicas only), so this reduction and
the barriers are all that the ranks share."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        out.put((rank, bench.max_over_ranks(times[rank], world, device="cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    times = [0.2251, 0.2317]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_rank, args=(2, _free_port(), times, q), nprocs=2, join=True, start_method="spawn")
    got = dict(q.get(timeout=60) for _ in range(2))
    assert got == {0: max(times), 1: max(times)}


def test_whole_job_value():
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    one = bench.whole_job_gbs(1_000_000_000, 0.25, 1)
    assert abs(one - 4000.0) < 1e-9
    assert abs(bench.whole_job_gbs(1_000_000_000, 0.25, 2) - 2 * one) < 1e-9

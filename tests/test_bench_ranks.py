"""The multi-rank timing logic of bench.py (weak scaling, one replica per GPU, no data-path
collective): two gloo ranks on the CPU each time a different amount, the job's time is the
slowest rank's, and rows/s counts the rows of every rank."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [40.0, 55.0][rank]
        slowest = bench.max_over_ranks(local_ms, world, device="cpu")
        rate = bench.weak_scaling_rate(1000, world, slowest / 1000.0)
        dist.barrier()
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_rows():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(2))
    for rank, slowest, rate in got:
        assert slowest == 55.0
        assert rate == pytest.approx(2 * 1000 / 0.055)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.weak_scaling_rate(262144, 1, 0.1) == pytest.approx(2621440.0)

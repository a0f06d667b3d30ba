"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Under torchrun every rank advances its own replica of the workload (independent tubes: weak scaling, no
collective on the data path); the job time is the slowest rank's, the value counts every rank's units, and
only rank 0 prints (and runs the CPU reference arm)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [1.5 + rank, 10.0 - rank]  # per-rank timings (seconds)
        red = bench.reduce_max_over_ranks(local, world, device="cpu")
        rate = bench.whole_job_rate(1_000_000, 10, world, red[0])
        out[rank] = (red, rate, bench.rank_prints(rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        red, rate, prints = out[rank]
        assert red == [2.5, 10.0]
        assert rate == pytest.approx(2 * 1_000_000 * 10 / 2.5 / 1e9)
        assert prints == (rank == 0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max_over_ranks([3.0], 1) == [3.0]
    assert bench.whole_job_rate(10, 2, 1, 4.0) == pytest.approx(5e-9)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 3, 2

    bench.run_reference(A, [], "none", rank=1)  # returns at once: no pool, no output
    assert capsys.readouterr().out == ""

"""The N > 1 bookkeeping of bench.py on CPU: two gloo ranks (the bench runs one
process per GPU, each advancing its own replica with no data collective)
agree on the slowest rank's timings, report the whole-job value, and only
rank 0 runs the oracle arm."""
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


def _rank_main(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank step time and end-to-end time: rank 1 is the slower one
        ms, e2e = (2.0, 0.5) if rank == 0 else (3.0, 0.25)
        got = bench.max_over_ranks([ms, e2e], dist, "cpu")
        value = bench.whole_job_value(1000, world, got[0] / 1e3)
        out[rank] = (got, value, bench.reference_rank_runs(rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        got, value, runs_ref = res[rank]
        assert got == [3.0, 0.5]                       # element-wise max over ranks
        assert value == pytest.approx(world * 1000 / 3e-3)
        assert runs_ref == (rank == 0)


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None, "cpu") == [1.5, 2.5]
    assert bench.whole_job_value(10, 1, 0.5) == 20.0

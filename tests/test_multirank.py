"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
runs its own replica of the workload, the job's time is the slowest rank's
(all_reduce MAX after a barrier) and rank 0 reports the whole-job value.
There is no data-path collective: the step does not shard on one GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 135.5][rank]
    dist.barrier()
    total = bench.max_over_ranks(local_ms, world)
    value = bench.job_value(1000, 4, world, total)
    q.put((rank, total, value))
    dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank_and_sums_the_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in out:
        assert total == 135.5
        assert value == pytest.approx(2 * 1000 * 4 / 0.1355)


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.job_value(10, 3, 1, 1000.0) == pytest.approx(30.0)

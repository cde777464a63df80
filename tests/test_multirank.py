"""The multi-rank path of bench.py on the CPU: two gloo ranks, each timing its own replica of
the workload; the job value is (ranks · steps) / the slowest rank's time."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        # rank r pretends its timed region took (1 + r) s and its e2e region (2 + r) s
        vals, mx = bench.aggregate_over_ranks([1.0 + rank, 2.0 + rank], steps=10, world=world)
        q.put((rank, vals, mx))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, vals, mx in out:
        assert mx == [2.0, 3.0]  # the slowest rank's seconds, on every rank
        assert vals == pytest.approx([2 * 10 / 2.0, 2 * 10 / 3.0])


def test_single_rank_aggregation():
    import bench

    vals, mx = bench.aggregate_over_ranks([0.5, 1.0], steps=4, world=1)
    assert vals == pytest.approx([8.0, 4.0]) and mx == [0.5, 1.0]

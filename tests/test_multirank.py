"""N > 1 bench logic on CPU with two gloo ranks: each rank times its own replica,
the job time is the maximum over ranks and the value counts every rank's work."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank
    m = bench.max_over_ranks(local_ms, dist, "cpu")
    v = bench.whole_job_value(1_000_000, 5, world, m)
    q.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == 150.0
        assert v == pytest.approx(2 * 1_000_000 * 5 / 0.150 / 1e9)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_value(4, 2, 1, 1000.0) == pytest.approx(8e-9)

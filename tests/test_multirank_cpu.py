"""World-size-2 checks of bench.py's multi-replica accounting on CPU (gloo):
the path shards into independent replicas, so the only cross-rank step is
the maximum of the per-rank times, and the job's throughput counts every
rank's iterations against the slowest rank's time."""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [100.0 + 50.0 * rank, 300.0 - 10.0 * rank]
    out = bench.max_over_ranks(times)
    q.put((rank, out, bench.job_throughput(world, 4, out[0])))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, out, thr in res:
        assert out == [150.0, 300.0]          # max of each entry over ranks
        assert thr == pytest.approx(2 * 4 / 0.150)

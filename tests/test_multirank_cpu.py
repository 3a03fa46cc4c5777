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


# --------------------------------------------------------------------------
# Row distribution of H|psi> (paper: Sparse State-Vector Emulation section,
# parallelisation paragraph): rows split uniformly over the processes, the
# state replicated, one collective per operation.  The exchange code of
# paper_2604_01176_gb300.shard runs here on gloo with each rank's block of
# sigma formed by the oracle (on a GPU, hy_apply_h_rows forms it).
# --------------------------------------------------------------------------
def test_row_split_covers_rows_once():
    from paper_2604_01176_gb300.shard import row_split
    for n_rows in (0, 1, 7, 35, 12870):
        for world in (1, 2, 3, 8):
            spans = [row_split(n_rows, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n_rows
            assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1


def _shard_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import oracle
    import synth
    from paper_2604_01176_gb300.shard import gather_blocks, reduce_partials, row_split
    n, na, nb, seed = 7, 3, 3, 77
    h1, h2, ec = synth.integrals(n, seed)
    ref = oracle.System(h1, h2, ec, n, na, nb)
    psi = synth.random_state(ref.n_det, 4)
    b, e = row_split(ref.n_astr, world, rank)
    rows = np.arange(b * ref.n_bstr, e * ref.n_bstr)
    block = torch.from_numpy(ref.sigma_rows(psi, rows) if len(rows) else np.zeros(0))
    full = gather_blocks(block, ref.n_astr, ref.n_bstr)
    part = torch.tensor([float(psi[rows] @ block.numpy())], dtype=torch.float64)
    e_tot = float(reduce_partials(part)[0])
    q.put((rank, full.numpy(), e_tot))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_blocks_all_gather_and_energy_all_reduce(world):
    import numpy as np
    import oracle
    import synth
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    h1, h2, ec = synth.integrals(7, 77)
    ref = oracle.System(h1, h2, ec, 7, 3, 3)      # 35 alpha rows: uneven blocks
    psi = synth.random_state(ref.n_det, 4)
    sig = ref.sigma(psi)
    for rank, full, e_tot in res:
        assert np.array_equal(full, sig)          # blocks reassembled in row order, bit for bit
        assert abs(e_tot - float(psi @ sig)) < 1e-12

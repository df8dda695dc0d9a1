"""The N > 1 benchmark path (replicas, no data-path collective) on CPU ranks:
two gloo processes agree on the slowest rank's time and on the whole-job
aggregate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [12.5, 20.0][rank]
    m = bench.max_over_ranks(local, torch.device("cpu"))
    q.put((rank, m, bench.aggregate_gpx_s(1000, 10, m, world)))
    dist.destroy_process_group()


def test_two_ranks_take_the_max_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [20.0, 20.0]
    assert all(abs(g[2] - 2 * 1000 * 10 / 0.020 / 1e9) < 1e-12 for g in got)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.0, torch.device("cpu")) == 3.0

"""Multi-GPU runs are replicas: each rank steps its own discharge (its own
seed) and the job's figures are the slowest rank's time and the pushes of all
ranks.  Two gloo ranks on the CPU run the benchmark's reduction and seeding
(the same functions the benchmark calls under torch.distributed.run)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as D  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    D.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        t_ms = [10.0, 12.5][rank]
        pushes = [100, 300][rank]
        t, n = bench.reduce_replicas(D, t_ms, pushes, "cpu")
        seeds = [None] * world
        D.all_gather_object(seeds, bench.replica_seed(1, rank))
        out.put((rank, t, n, seeds))
    finally:
        D.destroy_process_group()


def test_two_replicas_reduce_to_the_slowest_time_and_all_pushes():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n, seeds in res:
        assert t == 12.5            # the slowest rank
        assert n == 400.0           # every rank's pushes
        assert seeds == [1, 2]      # independent discharges

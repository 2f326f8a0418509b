"""The multi-rank path of bench.py (replicas only: no data-path collective,
a barrier and a max over ranks of the timed region) on CPU with gloo,
world size 2."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w, r, _ = bench.dist_env()
    # rank r pretends its timed region took 1 + r seconds for 10 units
    value, t = bench.job_throughput(10.0, 1.0 + r, w)
    dist.barrier()
    out.put((rank, w, r, value, t))
    dist.destroy_process_group()


def test_replicas_throughput_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, w, r, value, t in res:
        assert w == 2 and r == rank
        assert t == 2.0  # the slowest rank's time
        assert value == 10.0 * 2 / 2.0  # all ranks' units over the max time
    del torch


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.job_throughput(5.0, 2.0, 1) == (2.5, 2.0)

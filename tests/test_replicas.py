"""The replica (weak-scaling) host logic under a world_size-2 gloo process
group on CPU: the whole-job rate is the sum of the ranks' units over the
slowest rank's time."""

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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1607_01475_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = replicas.dist_env()
        units = 1000.0 * (rank + 1)        # rank 0: 1000, rank 1: 2000
        ms = 10.0 if rank == 0 else 40.0   # the slowest rank takes 40 ms
        rate, tmax = replicas.whole_job_rate(units, ms, dist)
        out.put((rank, r, w, lr, rate, tmax))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, r, w, lr, rate, tmax in res:
        assert (r, w, lr) == (rank, 2, rank)
        assert tmax == 40.0
        assert abs(rate - 3000.0 / 0.040) < 1e-6


def test_single_process_identity():
    from paper_1607_01475_gb300 import replicas
    rate, ms = replicas.whole_job_rate(500.0, 20.0, None)
    assert ms == 20.0 and abs(rate - 25000.0) < 1e-9

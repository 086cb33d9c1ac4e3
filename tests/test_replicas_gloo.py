"""The multi-GPU bench runs independent replicas; the only cross-rank step is the bookkeeping of
the whole-job numbers (slowest rank's time, states converged on all ranks). Checked here with
two gloo ranks on CPU."""
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


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, n = bench.aggregate_replicas(1.5 + rank, 70 + rank, dist)
    q.put((rank, t, n))
    dist.destroy_process_group()


def test_replica_bookkeeping_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n in res:
        assert t == 2.5 and n == 141


def test_single_process_is_identity():
    import bench
    assert bench.aggregate_replicas(3.0, 12, None) == (3.0, 12)

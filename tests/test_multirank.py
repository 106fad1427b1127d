"""Replicas on several ranks (bench.py --gpus N): the timed region is the maximum over
ranks and the cell updates are summed. World size 2 over gloo on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2502_08034_gb300 import workflows
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = workflows.reduce_over_ranks(dist, 100.0 + 50.0 * rank, 1000 * (rank + 1))
    q.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_reduce_max_time_and_sum_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u in out:
        assert t == 150.0 and u == 3000.0


def test_single_rank_passthrough():
    from paper_2502_08034_gb300 import workflows
    assert workflows.reduce_over_ranks(None, 12.5, 7) == (12.5, 7.0)

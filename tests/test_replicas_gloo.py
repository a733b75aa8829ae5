"""The multi-rank (replica) timing logic of bench.py with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2003_09956_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = replicas.rank_info()
    replicas.barrier(dist)
    t = 1.0 + 0.5 * r                     # rank 1 is the slow one
    tmax = replicas.max_over_ranks(dist, t)
    rate = replicas.aggregate_rate(w, 100.0, tmax)
    out.put((r, w, lr, tmax, rate))
    replicas.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
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
    assert [r[0] for r in res] == [0, 1]
    for r, w, lr, tmax, rate in res:
        assert w == 2 and lr == r
        assert tmax == pytest.approx(1.5)
        assert rate == pytest.approx(2 * 100.0 / 1.5)


def test_single_process_defaults():
    assert replicas.max_over_ranks(None, 3.25) == 3.25
    assert replicas.aggregate_rate(1, 10.0, 2.0) == 5.0

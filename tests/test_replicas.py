"""The multi-rank (replica) path on CPU: two gloo ranks, disjoint seeds,
max-reduction of timings and FP64 sums of observables (no GPU needed)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2102_05613_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = replicas.max_over_ranks(0.5 + rank, dist)
    s = replicas.sum_over_ranks([rank + 1.0, 10.0], dist)
    out[rank] = (t, s, replicas.seed_base(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 1.5
    assert out[0][1] == out[1][1] == [3.0, 20.0]
    assert out[0][2] != out[1][2]


def test_single_process_is_identity():
    assert replicas.max_over_ranks(2.5) == 2.5
    assert replicas.sum_over_ranks([1.0, 2.0]) == [1.0, 2.0]

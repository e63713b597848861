"""The replicated (N > 1) path of bench.py, on CPU with two gloo ranks: each
rank verifies its own batch, the job's time is the slowest rank's and its
pair count the sum over ranks; replicas draw different inputs."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [2.5, 4.0][rank]
    pairs = [1000, 3000][rank]
    e2e = [3.0, 5.5][rank]
    out = bench.combine_ranks(dist, ms, pairs, e2e, torch.device("cpu"))
    dist.barrier()
    q.put((rank, out))
    dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, pairs, e2e = res[r]
        assert ms == 4.0 and pairs == 4000 and e2e == 5.5     # max time, summed pairs
    assert 4000 / (4.0 / 1e3) == pytest.approx(1e6)


def test_single_rank_is_identity():
    assert bench.combine_ranks(None, 1.5, 10, 2.0, None) == (1.5, 10, 2.0)


def test_replicas_draw_their_own_inputs():
    w = bench.WORKLOADS["jaccard-small"]
    a, _ = bench.make_inputs(w, rank=0)
    b, _ = bench.make_inputs(w, rank=1)
    assert a.n == b.n
    assert not (len(a.indices) == len(b.indices) and (a.indices == b.indices).all())

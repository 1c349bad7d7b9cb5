"""The benchmark's multi-rank path on CPU: two gloo ranks, each an
independent replica; the job rate is all ranks' units over the slowest
rank's time (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000 + 10 * rank
    local_ms = 2.0 + rank            # rank 1 is the slowest
    max_ms, rate = bench.aggregate_ranks(units, local_ms, 5, dist, torch.device("cpu"))
    q.put((rank, max_ms, rate))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
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
    for rank, max_ms, rate in res:
        assert max_ms == pytest.approx(3.0)
        assert rate == pytest.approx((1000 + 1010) * 5 / 3.0e-3)

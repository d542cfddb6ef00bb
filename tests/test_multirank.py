"""The multi-rank bench path on CPU: two gloo ranks through bench.py's own
helpers (rendezvous from the environment, barrier, max over ranks)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, n, dist = bench.dist_init()
    assert (r, n) == (rank, ws) and dist is not None
    bench.barrier(dist)
    # each rank reports its own time; every rank must see the slowest
    out[rank] = bench.max_over_ranks(dist, 10.0 * (rank + 1))
    bench.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_maximum():
    ws = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert dict(out) == {0: 20.0, 1: 20.0}


def test_single_rank_needs_no_process_group():
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK") if k in os.environ}
    try:
        assert bench.dist_init() == (0, 1, None)
        assert bench.max_over_ranks(None, 3.5) == 3.5
    finally:
        os.environ.update(env)

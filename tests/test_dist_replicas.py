"""Multi-process host logic of bench.py on CPU (gloo, world size 2): every
rank gets its own replica seed, the job time is the max over ranks, and the
whole-job throughput counts the updates of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ws_, rank_, _ = bench.dist_env()
        seed = bench.replica_seed(11, rank_)
        t = 1.0 + rank_              # pretend rank r took 1 + r seconds
        tmax = bench.reduce_max(t, ws_)
        bench.barrier(ws_)
        q.put((rank_, seed, tmax))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in (0, 1)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in procs)
    assert [g[1] for g in got] == [11, 12]          # distinct replicas
    assert all(g[2] == 2.0 for g in got)             # max over ranks


def test_single_rank_defaults(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.reduce_max(3.5, 1) == 3.5

"""bench.py --gpus N runs N independent replicas (the path does not shard): the
ranks meet at barriers and rank 0 reports the slowest rank's time.  Checked with
two gloo ranks on the CPU (no GPU, no CUDA call)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), MGEIG_BENCH_BACKEND="gloo")
    import bench
    r, ws, local, dist = bench.dist_init()
    bench.barrier(dist)
    t = bench.max_over_ranks(dist, 1.0 + r, "cpu")     # rank r "took" 1 + r seconds
    bench.barrier(dist)
    out.put((r, ws, local, t))
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[:3] for x in res] == [(0, 2, 0), (1, 2, 1)]
    assert all(x[3] == 2.0 for x in res)


def test_single_process_needs_no_process_group(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench.dist_init() == (0, 1, 0, None)
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5

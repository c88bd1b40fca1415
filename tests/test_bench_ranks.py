"""The multi-rank path of bench.py on CPU (gloo, world size 2): replicas only,
so the one collective is the final reduction of the timing (the slowest
rank's time, the sum of the events); the reference arm runs on rank 0 alone
and the other ranks return without work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms, ev = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 1000.0 * (rank + 1), device="cpu")
    q.put((rank, ms, ev))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world_size_2():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_over_ranks(None, 2.5, 7) == (2.5, 7)


def test_reference_arm_only_on_rank_zero(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup, weights = 2, 1, 0, "fp32"
    assert bench.run_reference(A()) == 0  # returns before building anything

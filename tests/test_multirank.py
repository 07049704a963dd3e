"""The benchmark's multi-rank logic on CPU with gloo, world size 2: each rank
registers its own frames (distinct seeds), the step time is the slowest
rank's, and the reported rate counts every rank's work (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        local_time = 1.0 + rank          # rank 1 is the slower one
        slowest = bench.max_over_ranks(local_time, dist, "cpu")
        rate = bench.whole_job_rate(320, ws, slowest)
        out.put((r, ws, local, bench.rank_seed(1000, r), slowest, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
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
    (r0, ws0, l0, s0, t0, v0), (r1, ws1, l1, s1, t1, v1) = res
    assert (r0, r1) == (0, 1) and ws0 == ws1 == 2 and (l0, l1) == (0, 1)
    assert s0 != s1                      # distinct frames per rank
    assert t0 == t1 == 2.0               # both report the slowest rank's time
    assert v0 == v1 == pytest.approx(320 * 2 / 2.0)


def test_single_process_defaults(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(100, 1, 2.0) == 50.0

"""Multi-GPU runs are replicas: each rank takes its own frame and nothing crosses ranks on the data
path. These world_size-2 gloo tests on the CPU cover the host logic bench.py uses for N > 1: the
per-rank frames, the max-over-ranks step time and the whole-job aggregate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        f = bench.rank_frame("rgbd_120x160", r)
        my_ms = 1.0 + r                     # rank 1 is the slow one
        ms = bench.max_over_ranks(my_ms, w)
        val = bench.aggregate_mtri_s(f.n_triangles, w, ms)
        q.put((r, w, float(f.points[60, 80, 2]), ms, val, f.n_triangles))
    finally:
        dist.destroy_process_group()


def test_replicas_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [2, 2]
    assert res[0][2] != res[1][2]                       # each rank runs its own frame
    assert res[0][3] == res[1][3] == 2.0                # the slowest rank's time, on every rank
    ntri = res[0][5]
    assert abs(res[0][4] - ntri * 2 / 2e-3 / 1e6) < 1e-9


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_mtri_s(1_000_000, 1, 1.0) == 1000.0

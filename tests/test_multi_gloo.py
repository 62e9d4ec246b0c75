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


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun the oracle arm runs on rank 0 alone; every other rank exits 0 without work.
    The line carries the fields of the contract (impl, cpu_baseline, e2e with no copies)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "rgbd_120x160", "--gpus", "2",
           "--steps", "1", "--warmup", "3"]
    out = {}
    for rank in (0, 1):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
        r = subprocess.run(cmd, cwd=root, env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        out[rank] = [l for l in r.stdout.splitlines() if l.strip()]
    assert out[1] == []
    assert len(out[0]) == 1
    line = json.loads(out[0][0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["unit"] == "Mtri/s"
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "Mtri/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}

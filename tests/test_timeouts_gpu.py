"""Device-side timeouts on the GPU, without a fault: a self-test kernel makes one of the path's
bounded waits run out with a short limit (the grid barrier with a CTA that leaves without
arriving, or an mbarrier that nothing arms). The wait must give up, the sync call must report
PL3D_ERR_TIMEOUT once and clear the control words, and the next frame must match the oracle."""
import os
import time

import numpy as np
import pytest

import oracle
from oracle.compare import compare
import synth

pytestmark = pytest.mark.gpu

LIMIT_NS = 20_000_000   # 20 ms


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2007_12065_gb300 as pl3d
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.set_threads(os.cpu_count() or 1)
    ex = pl3d.PlaneExtractor(0)
    yield pl3d, ex, torch
    ex.close()


def _frame_matches_oracle(pl3d, torch, run):
    f = synth.depth_camera_scene(60, 100, seed=71, n_boxes=2, ramp=True)
    p = pl3d.make_params(**f.params)
    dev = run(f, p)
    ref = oracle.extract_planes(f.points, oracle.OracleParams(**f.params), f.dominant_normals)
    rep = compare(dev, ref, oracle.OracleParams(**f.params), f.H, f.W)
    assert rep["segments"] > 3


@pytest.mark.parametrize("kind", [1, 2])
def test_context_wait_gives_up_reports_and_recovers(env, kind):
    pl3d, ex, torch = env
    pl3d.pl3d_sync(ex.ctx)                       # nothing pending
    t0 = time.perf_counter()
    pl3d.pl3d_selftest_wait_timeout(ex.ctx, kind, LIMIT_NS)
    with pytest.raises(pl3d.PL3DError) as e:
        pl3d.pl3d_sync(ex.ctx)
    waited = time.perf_counter() - t0
    assert e.value.status == pl3d.PL3D_ERR_TIMEOUT
    assert LIMIT_NS * 1e-9 <= waited < 5.0      # gave up after the limit, not after 1 s per wait
    pl3d.pl3d_sync(ex.ctx)                       # reported once, then cleared

    def run(f, p):
        out = ex(torch.from_numpy(f.points).cuda(), p, f.dominant_normals, want_groups=True)
        pl3d.pl3d_sync(ex.ctx)
        return {k: v.cpu().numpy() for k, v in out.items()}

    _frame_matches_oracle(pl3d, torch, run)


def test_selftest_rejects_bad_arguments(env):
    pl3d, ex, torch = env
    for kind, lim in ((0, LIMIT_NS), (3, LIMIT_NS), (1, 10), (2, 10**11)):
        with pytest.raises(pl3d.PL3DError) as e:
            pl3d.pl3d_selftest_wait_timeout(ex.ctx, kind, lim)
        assert e.value.status == pl3d.PL3D_ERR_INVALID_ARG
    pl3d.pl3d_sync(ex.ctx)


@pytest.mark.parametrize("kind", [1, 2])
def test_static_wait_gives_up_reports_and_recovers(env, kind):
    """The allocation-free entry point keeps its error word in its fixed array: pl3d_static_sync
    reads it, reports the timeout once and clears the barrier words for the next call."""
    pl3d, ex, torch = env
    pl3d.pl3d_static_sync()
    pl3d.pl3d_selftest_wait_timeout(None, kind, LIMIT_NS)
    with pytest.raises(pl3d.PL3DError) as e:
        pl3d.pl3d_static_sync()
    assert e.value.status == pl3d.PL3D_ERR_TIMEOUT
    pl3d.pl3d_static_sync()

    def run(f, p):
        n = f.n_triangles
        out = dict(mask=torch.empty(n, dtype=torch.uint8, device="cuda"),
                   normals=torch.empty((n, 3), device="cuda"),
                   labels=torch.empty(n, dtype=torch.int32, device="cuda"))
        nd = f.dominant_normals
        pl3d.pl3d_extract_planes_static(torch.from_numpy(f.points).cuda(), f.H, f.W, p, nd, nd.shape[0],
                                        out["mask"], out["normals"], out["labels"])
        pl3d.pl3d_static_sync()
        return {k: v.cpu().numpy() for k, v in out.items()}

    _frame_matches_oracle(pl3d, torch, run)

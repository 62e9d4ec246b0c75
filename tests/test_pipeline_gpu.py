"""Pipelined host-buffer frames (pl3d_pipeline_*): every frame's outputs are bit for bit those of
the plain single-frame entry point, in any mix of sizes and depths; tickets, kept statuses and
argument checks; a device wait that gave up between frames is reported by the next frame and
cleared."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2007_12065_gb300 as pl3d
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = pl3d.pl3d_create(0)
    yield pl3d, ctx, torch
    pl3d.pl3d_destroy(ctx)


def _frames():
    out = []
    for i, (H, W) in enumerate([(120, 160), (64, 1024), (97, 131), (240, 320), (33, 250), (2, 2)]):
        if W >= 250:
            f = synth.lidar_scene(H, W, seed=700 + i)
        else:
            f = synth.depth_camera_scene(H, W, seed=700 + i, n_boxes=3, noise_sigma=0.004, nan_frac=0.03)
        params = dict(f.params)
        if i == 2:
            params.update(min_triangles=15)
        if i == 3:
            params.update(max_offset=0.03, lap_iters=7, bil_iters=4)
        out.append((f, params))
    return out


def _alone(env, f, params):
    pl3d, ctx, torch = env
    H, W = f.points.shape[:2]
    n = 2 * (H - 1) * (W - 1)
    m = torch.empty(n, dtype=torch.uint8, device="cuda")
    nr = torch.empty((n, 3), device="cuda")
    lb = torch.empty(n, dtype=torch.int32, device="cuda")
    pl3d.pl3d_extract_planes(ctx, torch.from_numpy(np.ascontiguousarray(f.points)).cuda(), H, W,
                             pl3d.make_params(**params), f.dominant_normals, f.dominant_normals.shape[0], m, nr, lb)
    torch.cuda.synchronize()
    return m.cpu(), nr.cpu(), lb.cpu()


def _host(torch, f):
    H, W = f.points.shape[:2]
    n = 2 * (H - 1) * (W - 1)
    pts = torch.from_numpy(np.ascontiguousarray(f.points)).pin_memory()
    return pts, (torch.full((n,), 9, dtype=torch.uint8).pin_memory(), torch.full((n, 3), 9.0).pin_memory(),
                 torch.full((n,), -9, dtype=torch.int32).pin_memory())


def _same(torch, got, want):
    m, nr, lb = got
    assert torch.equal(m, want[0])
    assert torch.equal(nr.view(torch.int32), want[1].view(torch.int32))   # NaNs in the same places
    assert torch.equal(lb, want[2])


@pytest.mark.parametrize("depth", [1, 2, 3, 5])
def test_frames_match_the_single_frame_path(env, depth):
    pl3d, _, torch = env
    frames = _frames()
    want = [_alone(env, f, p) for f, p in frames]
    pl = pl3d.pl3d_pipeline_create(0, max_points=max(f.points.shape[0] * f.points.shape[1] for f, _ in frames),
                                   depth=depth)
    try:
        order = [0, 1, 2, 3, 4, 5, 3, 1, 0, 4, 2, 2, 5, 3]
        bufs = [_host(torch, frames[i][0]) for i in order]
        tickets = []
        for k, i in enumerate(order):
            f, p = frames[i]
            H, W = f.points.shape[:2]
            tickets.append(pl3d.pl3d_pipeline_submit(pl, bufs[k][0], H, W, pl3d.make_params(**p), f.dominant_normals,
                                                     f.dominant_normals.shape[0], *bufs[k][1]))
        assert tickets == list(range(1, len(order) + 1))
        # the last frame first: earlier ones complete before it, their statuses are kept
        assert pl3d.pl3d_pipeline_wait(pl, tickets[-1]) == 0
        for t in tickets:
            assert pl3d.pl3d_pipeline_wait(pl, t) == 0
        for k, i in enumerate(order):
            _same(torch, bufs[k][1], want[i])
    finally:
        pl3d.pl3d_pipeline_destroy(pl)


def test_frames_waited_one_by_one_reuse_their_buffers(env):
    """Each frame waited for right after the next is submitted: one set of host buffers per
    frame in flight, reused."""
    pl3d, _, torch = env
    f, p = _frames()[3]
    want = _alone(env, f, p)
    H, W = f.points.shape[:2]
    pl = pl3d.pl3d_pipeline_create(0, max_points=H * W, depth=2)
    try:
        bufs = [_host(torch, f) for _ in range(2)]
        prev = None
        for k in range(9):
            b = bufs[k % 2]
            t = pl3d.pl3d_pipeline_submit(pl, b[0], H, W, pl3d.make_params(**p), f.dominant_normals,
                                          f.dominant_normals.shape[0], *b[1])
            if prev is not None:
                assert pl3d.pl3d_pipeline_wait(pl, prev[0]) == 0
                _same(torch, prev[1][1], want)
                for o in prev[1][1]:
                    o.fill_(7)
            prev = (t, b)
        assert pl3d.pl3d_pipeline_wait(pl, prev[0]) == 0
        _same(torch, prev[1][1], want)
    finally:
        pl3d.pl3d_pipeline_destroy(pl)


def test_arguments_and_tickets(env):
    pl3d, _, torch = env
    f, p = _frames()[0]
    H, W = f.points.shape[:2]
    with pytest.raises(pl3d.PL3DError):
        pl3d.pl3d_pipeline_create(0, max_points=H * W, depth=0)
    with pytest.raises(pl3d.PL3DError):
        pl3d.pl3d_pipeline_create(0, max_points=H * W, depth=17)
    with pytest.raises(pl3d.PL3DError):
        pl3d.pl3d_pipeline_create(0, max_points=3, depth=2)
    pl = pl3d.pl3d_pipeline_create(0, max_points=H * W - 1, depth=2)
    try:
        pts, outs = _host(torch, f)
        with pytest.raises(pl3d.PL3DError) as e:   # larger than max_points
            pl3d.pl3d_pipeline_submit(pl, pts, H, W, pl3d.make_params(**p), f.dominant_normals,
                                      f.dominant_normals.shape[0], *outs)
        assert e.value.status == pl3d.PL3D_ERR_INVALID_ARG
        g = synth.depth_camera_scene(60, 80, seed=3)
        gp = dict(g.params, max_offset=0.05)
        pts2, outs2 = _host(torch, g)
        with pytest.raises(pl3d.PL3DError) as e:   # seed-relative region growing needs a context
            pl3d.pl3d_pipeline_submit(pl, pts2, 60, 80, pl3d.make_params(**dict(gp, flags=pl3d.PL3D_FLAG_SEED_PTP)),
                                      g.dominant_normals, g.dominant_normals.shape[0], *outs2)
        assert e.value.status == pl3d.PL3D_ERR_UNSUPPORTED
        for bad in (0, 1):   # no ticket issued yet
            assert pl3d.pl3d_pipeline_status(pl, bad) == pl3d.PL3D_ERR_INVALID_ARG
        t = pl3d.pl3d_pipeline_submit(pl, pts2, 60, 80, pl3d.make_params(**g.params), g.dominant_normals,
                                      g.dominant_normals.shape[0], *outs2)
        assert t == 1
        assert pl3d.pl3d_pipeline_status(pl, 2) == pl3d.PL3D_ERR_INVALID_ARG
        assert pl3d.pl3d_pipeline_wait(pl, 1) == 0
        assert pl3d.pl3d_pipeline_wait(pl, 1) == 0   # kept
        _same(torch, outs2, _alone(env, g, g.params))
    finally:
        pl3d.pl3d_pipeline_destroy(pl)
    pl3d.pl3d_pipeline_destroy(None)


def test_timeout_between_frames_is_reported_and_cleared(env):
    """An mbarrier wait made to run out on the pipeline's context while no frame is in flight:
    the next frame reports PL3D_ERR_TIMEOUT (its results count as void), the word is cleared, and
    the frame after it is correct and reports PL3D_OK."""
    pl3d, _, torch = env
    f, p = _frames()[0]
    want = _alone(env, f, p)
    H, W = f.points.shape[:2]
    pl = pl3d.pl3d_pipeline_create(0, max_points=H * W, depth=2)
    try:
        bufs = [_host(torch, f) for _ in range(3)]
        prm = pl3d.make_params(**p)
        nd, K = f.dominant_normals, f.dominant_normals.shape[0]
        t1 = pl3d.pl3d_pipeline_submit(pl, bufs[0][0], H, W, prm, nd, K, *bufs[0][1])
        assert pl3d.pl3d_pipeline_wait(pl, t1) == 0
        ctx = pl3d.pl3d_pipeline_context(pl)
        assert ctx != 0
        pl3d.pl3d_selftest_wait_timeout(ctx, 2, 2_000_000)
        torch.cuda.synchronize()
        t2 = pl3d.pl3d_pipeline_submit(pl, bufs[1][0], H, W, prm, nd, K, *bufs[1][1])
        assert pl3d.pl3d_pipeline_status(pl, t2) == pl3d.PL3D_ERR_TIMEOUT
        assert pl3d.pl3d_pipeline_status(pl, t2) == pl3d.PL3D_ERR_TIMEOUT   # kept
        t3 = pl3d.pl3d_pipeline_submit(pl, bufs[2][0], H, W, prm, nd, K, *bufs[2][1])
        assert pl3d.pl3d_pipeline_wait(pl, t3) == 0
        _same(torch, bufs[2][1], want)
    finally:
        pl3d.pl3d_pipeline_destroy(pl)

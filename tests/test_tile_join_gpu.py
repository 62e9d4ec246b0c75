"""Segments across tile borders (Algorithm 5 over the twins of Algorithm 2), joined two ways.

The single-frame kernel joins each tile border inside its bilateral pass: the second of the
border's two tiles to finish its tile-local labels joins it, decided by a per-border counter
that each launch raises by two. The two-launch host-buffer call and the batch kernel join the
same borders in a merge phase after a grid barrier. Labels are canonical (the smallest GID of a
segment), so both ways must give the same labels bit for bit, under every tile height, with the
offset test and tri_min, on ragged frames, and on repeated calls whose frames and tile heights
change the counters' layout between calls.
"""
import pytest

import synth

pytestmark = pytest.mark.gpu

SHAPES = [(33, 66), (77, 130), (120, 160), (31, 1030), (240, 320)]


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2007_12065_gb300 as pl3d
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = pl3d.pl3d_create(0)
    yield pl3d, ctx, torch
    pl3d.pl3d_set_tuning(ctx, None)
    pl3d.pl3d_destroy(ctx)


def _frame(H, W, seed):
    return synth.depth_camera_scene(H, W, seed=seed, n_boxes=3, noise_sigma=0.004, nan_frac=0.03)


def _device(env, f, p):
    pl3d, ctx, torch = env
    n = 2 * (f.H - 1) * (f.W - 1)
    pts = torch.from_numpy(f.points).cuda()
    m = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    nr = torch.full((n, 3), 7.0, dtype=torch.float32, device="cuda")
    lb = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    pl3d.pl3d_extract_planes(ctx, pts, f.H, f.W, p, f.dominant_normals, f.dominant_normals.shape[0], m, nr, lb)
    assert pl3d.pl3d_sync(ctx) == 0
    return m.cpu(), nr.cpu(), lb.cpu()


def _host(env, f, p):
    pl3d, ctx, torch = env
    n = 2 * (f.H - 1) * (f.W - 1)
    hp = torch.from_numpy(f.points).pin_memory()
    hm = torch.full((n,), 7, dtype=torch.uint8).pin_memory()
    hn = torch.full((n, 3), 7.0, dtype=torch.float32).pin_memory()
    hl = torch.full((n,), -7, dtype=torch.int32).pin_memory()
    pl3d.pl3d_extract_planes_host(ctx, hp, f.H, f.W, p, f.dominant_normals, f.dominant_normals.shape[0], hm, hn, hl)
    assert pl3d.pl3d_sync(ctx) == 0
    return hm, hn, hl


def _same(a, b):
    assert a[0].equal(b[0])
    assert a[1].nan_to_num(7.0).equal(b[1].nan_to_num(7.0))
    assert a[2].equal(b[2])


@pytest.mark.parametrize("bil_tile_h", [0, 8, 16, 24])
@pytest.mark.parametrize("extra", [{}, dict(max_offset=0.02, min_triangles=5)])
def test_in_pass_join_matches_merge_phase(env, bil_tile_h, extra):
    pl3d, ctx, torch = env
    pl3d.pl3d_set_tuning(ctx, bil_tile_h=bil_tile_h)
    try:
        for i, (H, W) in enumerate(SHAPES):
            f = _frame(H, W, 700 + i)
            p = pl3d.make_params(**dict(f.params, **extra))
            d = _device(env, f, p)
            _same(d, _host(env, f, p))
            assert (d[2] >= 0).any()   # the frame has segments to join
    finally:
        pl3d.pl3d_set_tuning(ctx, None)


def test_counters_survive_changing_frames_and_tile_heights(env):
    """Each launch adds two to every border counter it uses, whatever frame came before: a call
    after frames of other shapes and tile heights still joins every border exactly once."""
    pl3d, ctx, torch = env
    frames = [_frame(H, W, 750 + i) for i, (H, W) in enumerate(SHAPES)]
    refs = {}
    try:
        for k in range(3):
            for j, f in enumerate(frames):
                th = (0, 8, 16, 24)[(j + k) % 4]
                pl3d.pl3d_set_tuning(ctx, bil_tile_h=th)
                p = pl3d.make_params(**f.params)
                out = _device(env, f, p)
                if j not in refs:
                    pl3d.pl3d_set_tuning(ctx, None)
                    refs[j] = _host(env, f, p)
                _same(out, refs[j])
    finally:
        pl3d.pl3d_set_tuning(ctx, None)

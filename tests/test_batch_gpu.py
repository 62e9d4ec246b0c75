"""Batches: many frames of uneven sizes in one persistent launch (a CUDA graph), and the launch
shapes of the autotuner. A batch computes exactly what the single-frame path computes, frame by
frame, so its outputs are compared bit for bit with pl3d_extract_planes_ex; a few frames are
also held to the FP64 oracle's bounds."""
import os

import numpy as np
import pytest

import oracle
from oracle.compare import compare
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2007_12065_gb300 as pl3d
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.set_threads(os.cpu_count() or 1)
    ctx = pl3d.pl3d_create(0)
    yield pl3d, ctx, torch
    pl3d.pl3d_destroy(ctx)


def _frames():
    """Uneven sizes (ragged tails, single tiles, W % 4 != 0 without TMA), both parameter sets,
    and per-frame variations of iterations (single-iteration Laplacian passes beside fused ones
    in the same pass), thresholds, offsets and tri_min."""
    out = []
    shapes = [(120, 160), (64, 1024), (2, 2), (33, 65), (97, 131), (240, 320), (5, 7), (128, 250), (48, 64),
              (31, 31), (61, 1021)]
    for i, (H, W) in enumerate(shapes):
        if W >= 250 and H <= 128:
            f = synth.lidar_scene(H, W, seed=900 + i)
        else:
            f = synth.depth_camera_scene(H, W, seed=900 + i, n_boxes=3, noise_sigma=0.004, nan_frac=0.03,
                                         hfov_deg=60.0)
        params = dict(f.params)
        if i % 4 == 1:
            params.update(min_triangles=20)
        if i % 5 == 2:
            params.update(max_offset=0.02)
        if i == 4:
            params.update(lap_iters=0)
        if i == 5:
            params.update(bil_iters=9, lap_iters=10)      # several passes of each filter
        if i == 8:
            params.update(bil_iters=0, max_edge=0.0)
        if i in (3, 10):
            params.update(lap_iters=1)                    # 64-row tiles, one displacement buffer
        out.append((f, params))
    return out


def _alloc(torch, H, W):
    n = 2 * (H - 1) * (W - 1)
    return dict(mask=torch.full((n,), 7, dtype=torch.uint8, device="cuda"),
                normals=torch.full((n, 3), 7.0, device="cuda"),
                labels=torch.full((n,), -7, dtype=torch.int32, device="cuda"),
                points=torch.full((H, W, 3), 7.0, device="cuda"),
                groups=torch.full((n,), 7, dtype=torch.uint8, device="cuda"))


def _single(env, pts, f, params):
    pl3d, ctx, torch = env
    H, W = f.points.shape[:2]
    o = _alloc(torch, H, W)
    pl3d.pl3d_extract_planes_ex(ctx, pts, H, W, pl3d.make_params(**params), f.dominant_normals,
                                f.dominant_normals.shape[0], o["mask"], o["normals"], o["labels"], o["points"],
                                o["groups"])
    return o


def _batch(env, frames, with_optional=True):
    pl3d, ctx, torch = env
    b = pl3d.Batch()
    outs, pts = [], []
    for f, params in frames:
        H, W = f.points.shape[:2]
        p = torch.from_numpy(np.ascontiguousarray(f.points)).cuda()
        o = _alloc(torch, H, W)
        b.add(p, H, W, pl3d.make_params(**params), f.dominant_normals, o["mask"], o["normals"], o["labels"],
              o["points"] if with_optional else None, o["groups"] if with_optional else None)
        outs.append(o)
        pts.append(p)
    return b, outs, pts


def _same(a, b, keys=("mask", "normals", "labels", "points", "groups")):
    import torch
    for k in keys:
        x, y = a[k], b[k]
        if x.dtype.is_floating_point:
            assert torch.equal(torch.isnan(x), torch.isnan(y)), k
            assert torch.equal(torch.nan_to_num(x, 0.0), torch.nan_to_num(y, 0.0)), k
        else:
            assert torch.equal(x, y), k


def test_batch_equals_single_frames_bit_for_bit(env):
    pl3d, ctx, torch = env
    frames = _frames()
    b, outs, pts = _batch(env, frames)
    pl3d.pl3d_extract_planes_batched(ctx, b)
    pl3d.pl3d_sync(ctx)
    for (f, params), o, p in zip(frames, outs, pts):
        _same(o, _single(env, p, f, params))
    pl3d.pl3d_sync(ctx)


@pytest.mark.parametrize("idx", [0, 1, 5, 6, 10])
def test_batch_frames_meet_the_oracle_bounds(env, idx):
    pl3d, ctx, torch = env
    frames = _frames()
    b, outs, _ = _batch(env, frames)
    pl3d.pl3d_extract_planes_batched(ctx, b)
    pl3d.pl3d_sync(ctx)
    f, params = frames[idx]
    dev = {k: v.cpu().numpy() for k, v in outs[idx].items()}
    op = oracle.OracleParams(**params)
    ref = oracle.extract_planes(f.points, op, f.dominant_normals)
    rep = compare(dev, ref, op, f.points.shape[0], f.points.shape[1])
    print(idx, f.points.shape[:2], rep)


def test_graph_replay_skips_identical_uploads(env):
    pl3d, ctx, torch = env
    frames = _frames()[:6]
    b, outs, _ = _batch(env, frames)
    pl3d.pl3d_extract_planes_batched(ctx, b)
    pl3d.pl3d_sync(ctx)
    first = [{k: v.clone() for k, v in o.items()} for o in outs]
    s0 = pl3d.pl3d_batch_stats(ctx)
    for o in outs:
        for v in o.values():
            v.fill_(3)
    for _ in range(3):
        pl3d.pl3d_extract_planes_batched(ctx, b)
    pl3d.pl3d_sync(ctx)
    s1 = pl3d.pl3d_batch_stats(ctx)
    assert s1["graph_launches"] == s0["graph_launches"] + 3
    assert s1["desc_uploads"] == s0["desc_uploads"]          # same batch: nothing re-uploaded
    for a, o in zip(first, outs):
        _same(a, o)


def test_batch_on_side_stream_and_timing(env):
    pl3d, ctx, torch = env
    frames = _frames()[:4]
    b, outs, pts = _batch(env, frames, with_optional=False)
    s = torch.cuda.Stream()
    pl3d.pl3d_set_timing(ctx, True)
    pl3d.pl3d_read_timing(ctx, reset=True)
    pl3d.pl3d_extract_planes_batched(ctx, b, stream=s)
    t = pl3d.pl3d_read_timing(ctx, reset=True)
    pl3d.pl3d_set_timing(ctx, False)
    s.synchronize()
    assert t["frame_kernel"][1] == 1 and t["frame_kernel"][0] > 0
    assert all(t[k][0] > 0 for k in ("laplacian", "bilateral", "label_merge", "label_flatten"))
    for (f, params), o, p in zip(frames, outs, pts):
        _same(o, _single(env, p, f, params), keys=("mask", "normals", "labels"))


@pytest.mark.parametrize("tun", [dict(lap_fuse=1), dict(bil_fuse=1), dict(lap_fuse=2, bil_fuse=2, ctas_per_sm=1),
                                 dict(ctas_per_sm=1), dict(lap_fuse=3, bil_fuse=1, ctas_per_sm=2),
                                 dict(lap_tile_h=16, bil_tile_h=16), dict(lap_tile_h=48, bil_tile_h=24),
                                 dict(lap_tile_h=64, bil_tile_h=8, lap_fuse=2), dict(lap_fuse=1, lap_tile_h=40)])
def test_tuning_never_changes_a_result(env, tun):
    pl3d, ctx, torch = env
    frames = _frames()
    b, ref_outs, pts = _batch(env, frames)
    pl3d.pl3d_set_tuning(ctx, None)
    pl3d.pl3d_extract_planes_batched(ctx, b)
    pl3d.pl3d_sync(ctx)
    ref = [{k: v.clone() for k, v in o.items()} for o in ref_outs]
    single_ref = _single(env, pts[0], *frames[0])
    pl3d.pl3d_set_tuning(ctx, **tun)
    try:
        assert pl3d.pl3d_get_tuning(ctx).as_dict() == dict(
            dict(lap_fuse=0, bil_fuse=0, ctas_per_sm=0, lap_tile_h=0, bil_tile_h=0), **tun)
        b2, outs, _ = _batch(env, frames)
        pl3d.pl3d_extract_planes_batched(ctx, b2)
        single = _single(env, pts[0], *frames[0])
        pl3d.pl3d_sync(ctx)
    finally:
        pl3d.pl3d_set_tuning(ctx, None)
    for a, o in zip(ref, outs):
        _same(a, o)
    _same(single_ref, single)


def test_autotuner_picks_a_candidate_and_keeps_results(env):
    pl3d, ctx, torch = env
    frames = [(synth.mixed_frame(H, W, seed=300 + i), None) for i, (H, W) in enumerate(synth.MIXED_SIZES)]
    frames = [(f, f.params) for f, _ in frames]
    b, outs, pts = _batch(env, frames, with_optional=False)
    try:
        tun, ms = pl3d.pl3d_autotune_batched(ctx, b, reps=2)
        assert ms > 0
        assert tun.ctas_per_sm in (1, 2) and tun.lap_fuse >= 1 and tun.bil_fuse >= 1
        assert pl3d.pl3d_get_tuning(ctx).as_dict() == tun.as_dict()
        print("autotuned", tun.as_dict(), f"{ms:.3f} ms")
    finally:
        pl3d.pl3d_set_tuning(ctx, None)
    for (f, params), o, p in zip(frames, outs, pts):
        _same(o, _single(env, p, f, params), keys=("mask", "normals", "labels"))


def test_mixed_size_batch_of_256(env):
    """The 256-frame mixed batch (sizes 120x160 .. 128x2048, both generators): every frame equals
    its single-frame result; two frames are held to the oracle."""
    pl3d, ctx, torch = env
    bases = {hw: synth.mixed_frame(*hw, seed=104_000 + i) for i, hw in enumerate(synth.MIXED_SIZES)}
    rng = np.random.default_rng(104)
    picks = rng.integers(0, len(synth.MIXED_SIZES), 256)
    frames = []
    for i, k in enumerate(picks):
        base = bases[synth.MIXED_SIZES[int(k)]]
        # a fresh per-frame copy: the same scene seen with other noise on the range
        pts = base.points.copy()
        r = np.random.default_rng(7000 + i)
        pts *= (1.0 + r.normal(0.0, 1e-3, pts.shape[:2] + (1,))).astype(np.float32)
        f = synth.Frame(points=pts, dominant_normals=base.dominant_normals, params=base.params,
                        surface_id=base.surface_id, surface_normals=base.surface_normals,
                        surface_group=base.surface_group, name=base.name, meta=base.meta)
        frames.append((f, f.params))
    b, outs, pts = _batch(env, frames, with_optional=False)
    pl3d.pl3d_extract_planes_batched(ctx, b)
    pl3d.pl3d_sync(ctx)
    for (f, params), o, p in zip(frames, outs, pts):
        _same(o, _single(env, p, f, params), keys=("mask", "normals", "labels"))
    for idx in (3, 200):
        f, params = frames[idx]
        dev = {k: v.cpu().numpy() for k, v in outs[idx].items() if k in ("mask", "normals", "labels")}
        op = oracle.OracleParams(**params)
        ref = oracle.extract_planes(f.points, op, f.dominant_normals, sensitivity=False)
        rep = compare(dev, ref, op, f.points.shape[0], f.points.shape[1])
        print(idx, f.points.shape[:2], rep)


def test_batch_argument_errors(env):
    pl3d, ctx, torch = env
    f = synth.depth_camera_scene(16, 16, seed=1, n_boxes=1)
    pts = torch.from_numpy(f.points).cuda()
    o = _alloc(torch, 16, 16)
    # mixed Laplacian kernel sizes in one batch
    b = pl3d.Batch()
    b.add(pts, 16, 16, pl3d.make_params(lap_kernel=3), f.dominant_normals, o["mask"], o["normals"], o["labels"])
    b.add(pts, 16, 16, pl3d.make_params(lap_kernel=5), f.dominant_normals, o["mask"], o["normals"], o["labels"])
    before = pl3d.pl3d_launch_count(ctx)
    with pytest.raises(pl3d.PL3DError) as e:
        pl3d.pl3d_extract_planes_batched(ctx, b)
    assert e.value.status == pl3d.PL3D_ERR_UNSUPPORTED
    # a frame without lap iterations does not constrain the kernel size
    b = pl3d.Batch()
    b.add(pts, 16, 16, pl3d.make_params(lap_kernel=5), f.dominant_normals, o["mask"], o["normals"], o["labels"])
    b.add(pts, 16, 16, pl3d.make_params(lap_iters=0, lap_kernel=3), f.dominant_normals, o["mask"], o["normals"],
          o["labels"])
    pl3d.pl3d_extract_planes_batched(ctx, b)
    # one invalid frame rejects the whole batch before anything is enqueued
    b = pl3d.Batch()
    b.add(pts, 16, 16, pl3d.make_params(), f.dominant_normals, o["mask"], o["normals"], o["labels"])
    b.add(pts, 16, 16, pl3d.make_params(bil_sigma_len=0.0), f.dominant_normals, o["mask"], o["normals"], o["labels"])
    n0 = pl3d.pl3d_launch_count(ctx)
    with pytest.raises(pl3d.PL3DError) as e:
        pl3d.pl3d_extract_planes_batched(ctx, b)
    assert e.value.status == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_launch_count(ctx) == n0
    assert n0 == before + 1
    # an empty batch does nothing
    pl3d.pl3d_extract_planes_batched(ctx, pl3d.Batch())
    assert pl3d.pl3d_launch_count(ctx) == n0
    pl3d.pl3d_sync(ctx)


def test_single_iteration_batch_runs_lap1_nodes(env):
    """Every frame at one Laplacian iteration (3 x 3): the Laplacian runs as a lap1_kernel node of
    the graph before the batch kernel. Results equal single frames bit for bit, the launch count
    includes the node, and the Laplacian phase time comes from the node's own stamps."""
    pl3d, ctx, torch = env
    frames = [(f, dict(p, lap_iters=1)) for f, p in _frames()]
    frames[4] = (frames[4][0], dict(frames[4][1], lap_iters=0))   # a frame without smoothing beside them
    b, outs, pts = _batch(env, frames)
    n0 = pl3d.pl3d_launch_count(ctx)
    pl3d.pl3d_set_timing(ctx, True)
    pl3d.pl3d_read_timing(ctx, reset=True)
    pl3d.pl3d_extract_planes_batched(ctx, b)
    t = pl3d.pl3d_read_timing(ctx, reset=True)
    pl3d.pl3d_set_timing(ctx, False)
    assert pl3d.pl3d_launch_count(ctx) == n0 + 2
    assert t["laplacian"][0] > 0 and t["bilateral"][0] > 0
    assert t["laplacian"][0] + t["bilateral"][0] <= 1.05 * t["frame_kernel"][0]
    for (f, params), o, p in zip(frames, outs, pts):
        _same(o, _single(env, p, f, params))
    pl3d.pl3d_sync(ctx)

"""The frame server: continuous batching over several sensors, admission by device memory, and
the same result for every request alone and in the mix (bit for bit: a batch runs the same
arithmetic as a single frame)."""
import time

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


def _sensors():
    """Five sensors of different sizes and parameter sets (one with tri_min, one with the
    plane-offset test)."""
    out = []
    for i, (H, W) in enumerate([(120, 160), (64, 1024), (97, 131), (240, 320), (33, 250)]):
        if W >= 250:
            f = synth.lidar_scene(H, W, seed=500 + i)
        else:
            f = synth.depth_camera_scene(H, W, seed=500 + i, n_boxes=3, noise_sigma=0.004, nan_frac=0.03)
        params = dict(f.params)
        if i == 2:
            params.update(min_triangles=15)
        if i == 3:
            params.update(max_offset=0.03)
        out.append((f, params))
    return out


def _host_out(torch, H, W):
    n = 2 * (H - 1) * (W - 1)
    return (torch.full((n,), 9, dtype=torch.uint8).pin_memory(), torch.full((n, 3), 9.0).pin_memory(),
            torch.full((n,), -9, dtype=torch.int32).pin_memory())


def _alone(env, f, params):
    """The request's result from the plain single-frame entry point."""
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


def _equal(torch, a, b):
    assert torch.equal(a[0], b[0])
    assert torch.equal(torch.isnan(a[1]), torch.isnan(b[1]))
    assert torch.equal(torch.nan_to_num(a[1], 0.0), torch.nan_to_num(b[1], 0.0))
    assert torch.equal(a[2], b[2])


def _serve(env, n_requests, seed, gap_s, **cfg):
    pl3d, ctx, torch = env
    sensors = _sensors()
    pts = [torch.from_numpy(np.ascontiguousarray(f.points)).pin_memory() for f, _ in sensors]
    srv = pl3d.pl3d_server_create(0, hbm_bytes=2 << 30, **cfg)
    rng = np.random.default_rng(seed)
    which = [int(rng.integers(0, len(sensors))) for _ in range(n_requests)]
    outs = [_host_out(torch, *sensors[s][0].points.shape[:2]) for s in which]     # pinned before the burst
    prm = [pl3d.make_params(**params) for _, params in sensors]
    reqs = {}
    try:
        for s, out in zip(which, outs):
            f = sensors[s][0]
            H, W = f.points.shape[:2]
            t = pl3d.pl3d_server_submit(srv, pts[s], H, W, prm[s], f.dominant_normals, f.dominant_normals.shape[0],
                                        *out)
            reqs[t] = (s, out)
            if gap_s:
                time.sleep(gap_s * rng.exponential())
        pl3d.pl3d_server_drain(srv)
        done = pl3d.pl3d_server_poll(srv, max_n=n_requests + 8)
        stats = pl3d.pl3d_server_get_stats(srv)
    finally:
        pl3d.pl3d_server_destroy(srv)
    return sensors, reqs, done, stats


def _check_all(env, sensors, reqs, done):
    pl3d, ctx, torch = env
    assert sorted(c["ticket"] for c in done) == sorted(reqs)
    assert all(c["status"] == 0 for c in done)
    assert all(c["latency_ms"] >= c["queue_ms"] >= 0 for c in done)
    alone = [_alone(env, f, params) for f, params in sensors]
    for t, (s, out) in reqs.items():
        _equal(torch, out, alone[s])


def test_served_results_equal_alone_and_batches_form(env):
    sensors, reqs, done, stats = _serve(env, 80, seed=1, gap_s=0.0, max_inflight=2, max_batch_frames=16)
    _check_all(env, sensors, reqs, done)
    print(stats)
    assert stats["completed"] == stats["submitted"] == 80
    assert stats["max_batch_frames"] > 1          # requests that waited were batched
    assert stats["batches"] < 80
    assert max(c["batch_frames"] for c in done) == stats["max_batch_frames"]


def test_served_with_poisson_gaps_two_in_flight(env):
    sensors, reqs, done, stats = _serve(env, 60, seed=2, gap_s=0.0003, max_inflight=2, max_batch_frames=8)
    _check_all(env, sensors, reqs, done)
    print(stats, np.percentile([c["latency_ms"] for c in done], [50, 99]))


def test_sequential_fifo_mode(env):
    sensors, reqs, done, stats = _serve(env, 25, seed=3, gap_s=0.0, max_inflight=1, max_batch_frames=1)
    _check_all(env, sensors, reqs, done)
    assert stats["max_batch_frames"] == 1 and stats["max_inflight"] == 1 and stats["batches"] == 25


def test_one_slot_batched_mode(env):
    sensors, reqs, done, stats = _serve(env, 30, seed=4, gap_s=0.0, max_inflight=1, max_batch_frames=64)
    _check_all(env, sensors, reqs, done)
    assert stats["max_inflight"] == 1


def test_admission_by_device_memory(env):
    pl3d, ctx, torch = env
    f = synth.depth_camera_scene(240, 320, seed=77, n_boxes=3)
    big = synth.depth_camera_scene(480, 640, seed=78, n_boxes=3)
    # a slot holds 72 B per pixel of buffers and scratch: room for one 240 x 320 frame, not two
    hbm = 2 * int(72 * 240 * 320 * 1.5)
    srv = pl3d.pl3d_server_create(0, max_inflight=2, max_batch_frames=16, hbm_bytes=hbm)
    try:
        p = torch.from_numpy(f.points).pin_memory()
        outs = {}
        for _ in range(6):
            o = _host_out(torch, 240, 320)
            outs[pl3d.pl3d_server_submit(srv, p, 240, 320, pl3d.make_params(**f.params), f.dominant_normals,
                                         f.dominant_normals.shape[0], *o)] = o
        with pytest.raises(pl3d.PL3DError) as e:
            pb = torch.from_numpy(big.points).pin_memory()
            pl3d.pl3d_server_submit(srv, pb, 480, 640, pl3d.make_params(**big.params), big.dominant_normals,
                                    big.dominant_normals.shape[0], *_host_out(torch, 480, 640))
        assert e.value.status == pl3d.PL3D_ERR_OUT_OF_MEMORY
        pl3d.pl3d_server_drain(srv)
        done = pl3d.pl3d_server_poll(srv)
        stats = pl3d.pl3d_server_get_stats(srv)
    finally:
        pl3d.pl3d_server_destroy(srv)
    assert len(done) == 6 and stats["rejected"] == 1 and stats["max_batch_frames"] == 1
    ref = _alone(env, f, f.params)
    for o in outs.values():
        _equal(torch, o, ref)


def test_poll_semantics_and_unsupported_two_slot_frame(env):
    pl3d, ctx, torch = env
    srv = pl3d.pl3d_server_create(0, max_inflight=2, max_batch_frames=4, hbm_bytes=1 << 30)
    try:
        assert pl3d.pl3d_server_poll(srv, wait_ms=0) == []
        assert pl3d.pl3d_server_poll(srv, wait_ms=-1) == []      # nothing outstanding: returns at once
        f = synth.depth_camera_scene(40, 48, seed=5, n_boxes=1)
        p = torch.from_numpy(f.points).pin_memory()
        # a 7 x 7 bilateral window over 16 iterations needs 150 KB of shared memory per CTA:
        # two batches of it cannot be resident side by side
        with pytest.raises(pl3d.PL3DError) as e:
            pl3d.pl3d_server_submit(srv, p, 40, 48, pl3d.make_params(bil_kernel=7, bil_iters=16),
                                    f.dominant_normals, f.dominant_normals.shape[0], *_host_out(torch, 40, 48))
        assert e.value.status == pl3d.PL3D_ERR_UNSUPPORTED
        o = _host_out(torch, 40, 48)
        t = pl3d.pl3d_server_submit(srv, p, 40, 48, pl3d.make_params(bil_kernel=7, bil_iters=2), f.dominant_normals,
                                    f.dominant_normals.shape[0], *o)
        got = pl3d.pl3d_server_poll(srv, wait_ms=-1)
        assert [c["ticket"] for c in got] == [t]
    finally:
        pl3d.pl3d_server_destroy(srv)
    _equal(torch, o, _alone(env, f, dict(pl3d.make_params(bil_kernel=7, bil_iters=2).as_dict())))


@pytest.mark.parametrize("max_inflight,max_batch", [(2, 64), (1, 1)])
def test_native_trace_replay(env, max_inflight, max_batch):
    """pl3d_server_replay submits a Poisson trace at its scheduled times from native code and
    reports the latency from each scheduled arrival. Every request completes without error; after
    the replay each ring set holds the result of the last request that used it, bit for bit the
    single-frame result of that request's frame."""
    pl3d, ctx, torch = env
    sens = _sensors()
    srv = pl3d.pl3d_server_create(0, max_inflight=max_inflight, max_batch_frames=max_batch, hbm_bytes=2 << 30)
    ring = 3
    sources = []
    for f, params in sens:
        H, W = f.points.shape[:2]
        variants = [f.points, (f.points * np.float32(1.001))]
        sources.append(dict(points=[torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in variants],
                            params=pl3d.make_params(**params), dominant_normals=f.dominant_normals,
                            outputs=[_host_out(torch, H, W) for _ in range(ring)]))
    rng = np.random.default_rng(7)
    n = 300
    arr = np.cumsum(rng.exponential(1.0 / 1500.0, n))
    which = rng.integers(0, len(sens), n)
    try:
        rep = pl3d.pl3d_server_replay(srv, sources, arr, which)
    finally:
        pl3d.pl3d_server_destroy(srv)
    print(rep)
    assert rep["requests"] == n and rep["completed"] == n and rep["failed"] == 0
    assert 0 < rep["p50_ms"] <= rep["p90_ms"] <= rep["p99_ms"] <= rep["max_ms"]
    assert rep["seconds"] >= arr[-1] and rep["achieved_fps"] > 0 and rep["mtri_s"] > 0
    if max_batch == 1:
        assert rep["max_batch_frames"] == 1
    for s, (f, params) in enumerate(sens):
        ks = np.nonzero(which == s)[0]
        for k_set in range(ring):
            uses = [k for k in range(len(ks)) if k % ring == k_set]
            if not uses:
                continue
            variant = uses[-1] % 2
            g = synth.Frame(points=sources[s]["points"][variant].numpy(), dominant_normals=f.dominant_normals,
                            params=f.params, surface_id=f.surface_id, surface_normals=f.surface_normals,
                            surface_group=f.surface_group, name=f.name, meta=f.meta)
            want = _alone(env, g, params)
            got = sources[s]["outputs"][k_set]
            assert torch.equal(got[0], want[0]) and torch.equal(got[2], want[2])
            assert torch.equal(got[1].nan_to_num(7.0), want[1].nan_to_num(7.0))

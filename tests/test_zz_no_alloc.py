"""The allocation-free entry point against the context entry point, two calls in a row.

Some callers cannot allocate device memory while they run: a real-time sensor loop that must
not hit the device-wide synchronisation cudaMalloc/cudaFree can cause, a process whose memory
budget is fixed at start-up, or a plugin that gets a stream and buffers per call and keeps no
context. pl3d_extract_planes_static serves them with scratch from a fixed device array. Its
results must match pl3d_extract_planes within the parity tolerances (masks and labels exact,
normals within 1e-4 rad), and a second call must not see anything left over from the first.
This file is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _angle(a, b):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cr, np.einsum("ij,ij->i", a, b))


def _both(pl3d, torch, ctx, frame, params):
    H, W = frame.H, frame.W
    n = 2 * (H - 1) * (W - 1)
    nd = frame.dominant_normals
    pts = torch.from_numpy(frame.points).cuda()
    outs = []
    for static in (False, True):
        m = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        nrm = torch.full((n, 3), 7.0, dtype=torch.float32, device="cuda")
        lab = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        if static:
            pl3d.pl3d_extract_planes_static(pts, H, W, params, nd, nd.shape[0], m, nrm, lab)
        else:
            pl3d.pl3d_extract_planes(ctx, pts, H, W, params, nd, nd.shape[0], m, nrm, lab)
        torch.cuda.synchronize()
        outs.append((m.cpu().numpy(), nrm.cpu().numpy(), lab.cpu().numpy()))
    (m0, n0, l0), (m1, n1, l1) = outs
    assert np.array_equal(m0, m1)
    assert np.array_equal(l0, l1)
    nan0, nan1 = np.isnan(n0[:, 0]), np.isnan(n1[:, 0])
    assert np.array_equal(nan0, nan1)
    assert (_angle(n0[~nan0], n1[~nan0]) <= 1e-4).all()
    return l1


def test_static_entry_matches_context_entry_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2007_12065_gb300 as pl3d
    ctx = pl3d.pl3d_create(0)
    try:
        big = synth.rgbd_480x640()                       # the largest frame the fixed scratch holds
        small = synth.depth_camera_scene(90, 130, seed=31, n_boxes=3, ramp=True)
        la = _both(pl3d, torch, ctx, big, pl3d.make_params(**big.params))
        lb = _both(pl3d, torch, ctx, small, pl3d.make_params(**dict(small.params, min_triangles=20)))
        assert (la >= 0).sum() > 1000 and (lb >= 0).sum() > 100
        assert pl3d.pl3d_static_scratch_bytes() < 16 << 20
        # larger than the fixed scratch: rejected before anything is enqueued
        H, W = 481, 640
        n = 2 * (H - 1) * (W - 1)
        with pytest.raises(pl3d.PL3DError) as e:
            pl3d.pl3d_extract_planes_static(torch.zeros((H, W, 3), device="cuda"), H, W, pl3d.make_params(),
                                            np.array([[0, 0, 1]], np.float32), 1,
                                            torch.empty(n, dtype=torch.uint8, device="cuda"),
                                            torch.empty((n, 3), device="cuda"),
                                            torch.empty(n, dtype=torch.int32, device="cuda"))
        assert e.value.status == pl3d.PL3D_ERR_INVALID_ARG
        pl3d.pl3d_static_sync()                          # no device-side error was recorded
    finally:
        pl3d.pl3d_destroy(ctx)


def test_static_entry_allocates_nothing_and_keeps_its_bilateral_limit():
    """Once the first call has loaded the library's device code (and with it the fixed array),
    later calls leave the device's free memory unchanged. The fixed scratch has no carry buffers,
    so a kernel-3 bilateral runs at most 6 iterations (one tile pass): 6 is accepted and matches
    the context entry point, 7 is refused before anything is enqueued."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2007_12065_gb300 as pl3d
    f = synth.depth_camera_scene(120, 160, seed=33, n_boxes=3, ramp=True)
    H, W, n = f.H, f.W, f.n_triangles
    nd = f.dominant_normals
    pts = torch.from_numpy(f.points).cuda()
    outs = [(torch.empty(n, dtype=torch.uint8, device="cuda"), torch.empty((n, 3), device="cuda"),
             torch.empty(n, dtype=torch.int32, device="cuda")) for _ in range(2)]
    p6 = pl3d.make_params(**dict(f.params, bil_iters=6))
    pl3d.pl3d_extract_planes_static(pts, H, W, p6, nd, nd.shape[0], *outs[0])
    pl3d.pl3d_static_sync()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        pl3d.pl3d_extract_planes_static(pts, H, W, p6, nd, nd.shape[0], *outs[1])
        pl3d.pl3d_static_sync()
    assert torch.cuda.mem_get_info()[0] == free0
    assert all(torch.equal(a.nan_to_num(7.0), b.nan_to_num(7.0)) for a, b in zip(*outs))
    ctx = pl3d.pl3d_create(0)
    try:
        _both(pl3d, torch, ctx, f, p6)
    finally:
        pl3d.pl3d_destroy(ctx)
    with pytest.raises(pl3d.PL3DError) as e:
        pl3d.pl3d_extract_planes_static(pts, H, W, pl3d.make_params(**dict(f.params, bil_iters=7)), nd,
                                        nd.shape[0], *outs[1])
    assert e.value.status == pl3d.PL3D_ERR_INVALID_ARG

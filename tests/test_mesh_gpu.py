"""Explicit mesh (Algorithm 1: T, T_map; Algorithm 2: HE) and the segments' triangle lists and
boundary half-edges (the inputs of polygon extraction, Section 7.2) through pl3d_extract_mesh,
compared bit for bit with the oracle. Both sides take the same labels, computed by the oracle."""
import numpy as np
import pytest

import oracle
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


def _check(env, points, labels):
    pl3d, ctx, torch = env
    pts = torch.from_numpy(np.ascontiguousarray(points, dtype=np.float32)).cuda()
    lab = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.int32)).cuda() if labels is not None else None
    dev = pl3d.extract_mesh(ctx, pts, lab)
    ref = oracle.mesh_outputs(points, labels if labels is not None else np.full(
        2 * (points.shape[0] - 1) * (points.shape[1] - 1), -1, np.int32))
    assert dev["counts"][0] == len(ref["T"])
    assert np.array_equal(dev["T"].cpu().numpy(), ref["T"])
    assert np.array_equal(dev["Tmap"].cpu().numpy(), ref["Tmap"])
    assert np.array_equal(dev["HE"].cpu().numpy(), ref["HE"])
    if labels is not None:
        assert dev["counts"][1] == len(ref["seg_labels"]) and dev["counts"][2] == len(ref["seg_tris"])
        assert np.array_equal(dev["seg_labels"].cpu().numpy(), ref["seg_labels"])
        assert np.array_equal(dev["seg_offsets"].cpu().numpy(), ref["seg_offsets"])
        assert np.array_equal(dev["seg_tris"].cpu().numpy(), ref["seg_tris"])
        assert np.array_equal(dev["border"].cpu().numpy(), ref["border"])
    return dev, ref


def _oracle_labels(f, **kw):
    op = oracle.OracleParams(**dict(f.params, **kw))
    return oracle.extract_planes(f.points, op, f.dominant_normals, sensitivity=False)["labels"]


@pytest.mark.parametrize("name", ["rgbd_120x160", "rgbd_480x640", "lidar_64x1024"])
def test_mesh_and_segments_match_oracle(env, name):
    f = synth.WORKLOADS[name]()
    dev, ref = _check(env, f.points, _oracle_labels(f))
    print(name, dev["counts"])
    assert dev["counts"][1] > 10


@pytest.mark.parametrize("H,W", [(2, 2), (2, 3), (3, 2), (5, 7), (33, 65), (47, 129), (64, 2048 + 5)])
def test_ragged_shapes_and_chunk_borders(env, H, W):
    f = synth.depth_camera_scene(H, W, seed=H * 31 + W, n_boxes=2, noise_sigma=0.003, nan_frac=0.1, hfov_deg=40.0)
    _check(env, f.points, _oracle_labels(f, lap_iters=2, bil_iters=2))


def test_no_labels_and_all_invalid(env):
    f = synth.depth_camera_scene(40, 50, seed=3, n_boxes=1, nan_frac=0.2)
    _check(env, f.points, None)
    nanpts = np.full((20, 30, 3), np.nan, np.float32)
    dev, _ = _check(env, nanpts, np.full(2 * 19 * 29, -1, np.int32))
    assert dev["counts"] == (0, 0, 0)


def test_tri_min_and_offset_labels(env):
    f = synth.rgbd_120x160()
    _check(env, f.points, _oracle_labels(f, min_triangles=30))
    _check(env, f.points, _oracle_labels(f, max_offset=0.02))


def test_many_segments_three_radix_passes(env):
    """One segment per quad (label = the quad's first GID when both triangles are valid): about
    300,000 segments, so the sort runs three passes of 7-bit digits."""
    f = synth.rgbd_480x640()
    H, W = f.points.shape[:2]
    valid = np.isfinite(f.points).all(-1)
    Hq, Wq = H - 1, W - 1
    q = np.arange(Hq * Wq)
    u, v = q // Wq, q % Wq
    both = valid[u, v] & valid[u, v + 1] & valid[u + 1, v + 1] & valid[u + 1, v]
    labels = np.full(2 * Hq * Wq, -1, np.int32)
    labels[2 * q[both]] = 2 * q[both]
    labels[2 * q[both] + 1] = 2 * q[both]
    dev, ref = _check(env, f.points, labels)
    assert dev["counts"][1] > 65536


@pytest.mark.parametrize("n_seg", [1, 2, 255, 256, 2047, 2048, 2049, 4097])
def test_segment_counts_around_the_counting_pass(env, n_seg):
    """Up to 2048 segments the lists come from one counting pass, beyond it from the radix sort:
    n_seg - 1 segments of a single valid triangle, spread over the frame, and one segment of all
    other valid triangles (its label the smallest of their GIDs), on both sides of that limit."""
    f = synth.rgbd_120x160()
    _, Tmap = oracle.extract_triangles(oracle.widen(f.points))
    valid = np.nonzero(np.asarray(Tmap) >= 0)[0]
    single = valid[np.linspace(0, len(valid) - 1, n_seg - 1).astype(np.int64)] if n_seg > 1 else valid[:0]
    labels = np.full(len(Tmap), -1, np.int32)
    rest = np.setdiff1d(valid, single)
    labels[rest] = rest.min()
    labels[single] = single
    dev, ref = _check(env, f.points, labels)
    assert dev["counts"][1] == n_seg


def test_argument_checks(env):
    pl3d, ctx, torch = env
    import ctypes
    L = pl3d.lib()
    one = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = one.data_ptr()
    assert L.pl3d_extract_mesh(ctx, p, None, 1, 5, p, p, p, p, None, None, None, None, None) == pl3d.PL3D_ERR_INVALID_ARG
    # half-edge ids must fit int32: 6 (H-1)(W-1) >= 2^31
    assert L.pl3d_extract_mesh(ctx, p, None, 20000, 20000, p, p, p, p, None, None, None, None,
                               None) == pl3d.PL3D_ERR_INVALID_ARG
    # labels without segment buffers
    assert L.pl3d_extract_mesh(ctx, p, p, 4, 4, p, p, p, p, None, None, None, None, None) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_extract_mesh(None, p, None, 4, 4, p, p, p, p, None, None, None, None,
                               None) == pl3d.PL3D_ERR_INVALID_ARG

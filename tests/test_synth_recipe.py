"""The seeded input generators keep the recipe the design states for the paper's stand-in
workloads: sizes, FP32 layout, missing-point fractions, range noise and outliers measured
against each pixel's ground-truth plane, dominant normals that match the surfaces' groups, and
determinism per seed. Inputs only: none of the method's arithmetic is involved."""
import numpy as np
import pytest

import synth


def _residuals(f):
    """Distance of every valid point from its ground-truth surface plane (the plane's offset taken
    as the median over its pixels)."""
    P = f.points.reshape(-1, 3).astype(np.float64)
    s = f.surface_id.reshape(-1)
    ok = ~np.isnan(P[:, 0]) & (s >= 0)
    out = []
    for k in np.unique(s[ok]):
        m = ok & (s == k)
        d = P[m] @ f.surface_normals[k]
        out.append(d - np.median(d))
    return np.concatenate(out)


def _robust_sigma(r):
    return 1.4826 * np.median(np.abs(r - np.median(r)))


@pytest.fixture(scope="module")
def frames():
    return {name: fn() for name, fn in synth.WORKLOADS.items()}


@pytest.mark.parametrize("name,shape,k,nan_lo,nan_hi", [
    ("rgbd_120x160", (120, 160), 3, 0.015, 0.025),
    ("rgbd_480x640", (480, 640), 4, 0.025, 0.035),
    ("lidar_64x1024", (64, 1024), 2, 0.08, 0.14),
])
def test_shapes_missing_points_and_dominant_normals(frames, name, shape, k, nan_lo, nan_hi):
    f = frames[name]
    assert f.points.shape == shape + (3,) and f.points.dtype == np.float32 and f.points.flags["C_CONTIGUOUS"]
    nan = np.isnan(f.points).any(-1)
    assert np.array_equal(nan, np.isnan(f.points).all(-1))       # a missing point has no coordinate
    assert nan_lo < nan.mean() < nan_hi
    assert np.array_equal(nan, f.surface_id < 0)
    assert f.dominant_normals.shape == (k, 3)
    np.testing.assert_allclose(np.linalg.norm(f.dominant_normals, axis=1), 1.0, atol=1e-6)
    # every surface with a group lies along that group's dominant normal
    g = f.surface_group
    assert set(np.unique(g)) == set(range(k)) | {-1}
    dots = np.einsum("ij,ij->i", f.surface_normals[g >= 0], f.dominant_normals[g[g >= 0]].astype(np.float64))
    assert dots.min() > 0.999


def test_depth_noise_and_outliers(frames):
    r = _residuals(frames["rgbd_120x160"])
    assert 2e-3 < _robust_sigma(r) < 5.5e-3            # 5 mm along the ray, projected on the plane normal
    assert np.abs(r).max() < 0.05                       # no outliers at 120 x 160
    r = _residuals(frames["rgbd_480x640"])
    assert 2e-3 < _robust_sigma(r) < 5.5e-3
    assert 0.004 < (np.abs(r) > 0.05).mean() < 0.012    # 1% range outliers of up to 0.3 m


def test_lidar_noise_and_range(frames):
    f = frames["lidar_64x1024"]
    r = _residuals(f)
    assert 5e-3 < _robust_sigma(r) < 2.2e-2            # 2 cm along the ray
    P = f.points[~np.isnan(f.points[..., 0])].astype(np.float64)
    assert np.linalg.norm(P[:, :2], axis=1).max() < 100.5    # returns beyond 100 m are missing
    assert f.params["max_edge"] == 0.5 and f.params["lap_iters"] == 3 and f.params["bil_iters"] == 2


def test_depth_parameters(frames):
    for name in ("rgbd_120x160", "rgbd_480x640"):
        p = frames[name].params
        assert (p["lap_kernel"], p["lap_lambda"], p["lap_iters"]) == (3, 1.0, 5)
        assert (p["bil_kernel"], p["bil_sigma_len"], p["bil_sigma_ang"], p["bil_iters"]) == (3, 0.1, 0.15, 3)
        assert (p["min_dot"], p["max_edge"]) == (0.95, 0.1)


def test_generators_are_deterministic_per_seed():
    a, b = synth.rgbd_120x160(), synth.rgbd_120x160()
    assert np.array_equal(a.points, b.points, equal_nan=True)
    c = synth.rgbd_120x160(seed=7)
    assert not np.array_equal(a.points, c.points, equal_nan=True)
    m1, m2 = synth.mixed_frame(64, 1024, seed=5), synth.mixed_frame(64, 1024, seed=5)
    assert np.array_equal(m1.points, m2.points, equal_nan=True)
    assert synth.mixed_frame(240, 320, seed=5).points.shape == (240, 320, 3)

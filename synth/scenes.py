"""Seeded synthetic organized point clouds (inputs only; none of the method's arithmetic).

Two sensors stand in for the paper's RealSense, SynPEB and KITTI recordings, none of
which is available here:

* ``depth_camera_scene`` -- a pinhole depth camera in a room corner: floor z = 0, two
  walls (x = 3 m, y = 3 m), axis-aligned boxes on the floor, optionally a ramp tilted by
  15 degrees; Gaussian range noise along each ray, uniform range outliers and a fraction
  of pixels set to NaN (missing depth).
* ``lidar_scene`` -- a spinning LiDAR on a street: road z = 0, sidewalks raised by a curb,
  two building facades, car-sized boxes; range noise, missing returns, NaN beyond the
  maximum range.

Both ray-cast in FP64 and return FP32 xyz in a world frame (z up). Rows run downward in
the image and columns run to the right as seen from the sensor, so the right-hand rule
over the mesh's listed vertex order gives normals that face the sensor; the dominant
normals returned follow that convention.

Every frame also carries its ground truth: the id of the surface each pixel hit and each
surface's plane normal and dominant-normal group.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Frame:
    points: np.ndarray                  # float32 [H, W, 3], NaN = missing
    dominant_normals: np.ndarray        # float32 [K, 3]
    params: dict                        # method parameters (paper names)
    surface_id: np.ndarray              # int32 [H, W], -1 = no return / NaN
    surface_normals: np.ndarray         # float64 [S, 3], facing the sensor
    surface_group: np.ndarray           # int32 [S], index into dominant_normals or -1
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def H(self) -> int:
        return int(self.points.shape[0])

    @property
    def W(self) -> int:
        return int(self.points.shape[1])

    @property
    def n_triangles(self) -> int:
        return 2 * (self.H - 1) * (self.W - 1)


# ----------------------------------------------------------------------------- ray casting


class _Surfaces:
    """Accumulates nearest hits of a bundle of rays against planar patches and boxes."""

    def __init__(self, origin: np.ndarray, dirs: np.ndarray):
        self.o = origin.astype(np.float64)
        self.d = dirs.astype(np.float64)                       # [n, 3] unit
        n = dirs.shape[0]
        self.t = np.full(n, np.inf)
        self.sid = np.full(n, -1, np.int32)
        self.normals: list[np.ndarray] = []

    def _new(self, normal) -> int:
        self.normals.append(np.asarray(normal, np.float64) / np.linalg.norm(normal))
        return len(self.normals) - 1

    def _take(self, t, hit, sid):
        closer = hit & (t > 1e-9) & (t < self.t)
        self.t = np.where(closer, t, self.t)
        self.sid = np.where(closer, sid, self.sid)

    def axis_plane(self, axis: int, value: float, normal, bounds) -> int:
        """Patch of the plane coord[axis] = value, limited by bounds[(a, lo, hi)] on other axes."""
        sid = self._new(normal)
        dd = self.d[:, axis]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (value - self.o[axis]) / dd
        hit = np.isfinite(t) & (t > 0)
        with np.errstate(invalid="ignore"):
            p = self.o[None, :] + np.where(hit, t, 0.0)[:, None] * self.d
        for a, lo, hi in bounds:
            hit &= (p[:, a] >= lo) & (p[:, a] <= hi)
        self._take(t, hit, sid)
        return sid

    def box(self, lo, hi) -> list[int]:
        """Axis-aligned box; each of the five faces other than the bottom is its own surface."""
        lo = np.asarray(lo, np.float64)
        hi = np.asarray(hi, np.float64)
        ids = []
        for axis in range(3):
            others = [a for a in range(3) if a != axis]
            for side, value in ((-1, lo[axis]), (+1, hi[axis])):
                if axis == 2 and side == -1:
                    continue  # bottom face rests on the floor
                nrm = np.zeros(3)
                nrm[axis] = side
                ids.append(self.axis_plane(axis, value, nrm, [(a, lo[a], hi[a]) for a in others]))
        return ids

    def rect(self, p0, a_dir, b_dir, a_len, b_len, normal) -> int:
        """Planar rectangle p0 + s a + t b, s in [0, a_len], t in [-b_len/2, b_len/2]."""
        sid = self._new(normal)
        n = self.normals[sid]
        denom = self.d @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            t = ((np.asarray(p0) - self.o) @ n) / denom
        hit = np.isfinite(t) & (t > 0)
        p = self.o[None, :] + np.where(hit, t, 0.0)[:, None] * self.d - np.asarray(p0)[None, :]
        s = p @ np.asarray(a_dir)
        q = p @ np.asarray(b_dir)
        hit &= (s >= 0) & (s <= a_len) & (np.abs(q) <= b_len / 2)
        self._take(t, hit, sid)
        return sid


def _finish(surf: _Surfaces, rng, H, W, noise_sigma, outlier_frac, outlier_range, nan_frac, max_range):
    n = H * W
    t = surf.t.copy()
    sid = surf.sid.copy()
    valid = np.isfinite(t)
    t = t + rng.normal(0.0, noise_sigma, n)
    if outlier_frac > 0:
        out = rng.random(n) < outlier_frac
        t = np.where(out, t + rng.uniform(-outlier_range, outlier_range, n), t)
    drop = rng.random(n) < nan_frac
    valid &= ~drop
    if max_range is not None:
        valid &= t <= max_range
    valid &= t > 0
    pts = surf.o[None, :] + np.where(valid, t, 0.0)[:, None] * surf.d
    pts[~valid] = np.nan
    sid[~valid] = -1
    return pts.reshape(H, W, 3).astype(np.float32), sid.reshape(H, W)


# ----------------------------------------------------------------------------- depth camera

DEPTH_PARAMS = dict(lap_iters=5, lap_lambda=1.0, lap_kernel=3, bil_iters=3, bil_sigma_len=0.1, bil_sigma_ang=0.15,
                    bil_kernel=3, max_edge=0.1, min_dot=0.95, max_offset=0.0, min_triangles=0)


def depth_camera_scene(H: int = 120, W: int = 160, seed: int = 101, n_boxes: int = 4, ramp: bool = False,
                       noise_sigma: float = 0.005, outlier_frac: float = 0.0, outlier_range: float = 0.3,
                       nan_frac: float = 0.02, hfov_deg: float = 70.0, cam_height: float = 1.5,
                       yaw_deg: float = 45.0, pitch_deg: float = 30.0, wall: float = 3.0,
                       params: dict | None = None) -> Frame:
    rng = np.random.default_rng(seed)
    yaw, pitch = np.radians(yaw_deg), np.radians(pitch_deg)
    f = np.array([np.cos(yaw) * np.cos(pitch), np.sin(yaw) * np.cos(pitch), -np.sin(pitch)])
    r = np.array([np.sin(yaw), -np.cos(yaw), 0.0])
    d = np.cross(f, r)                                   # image "down"; (r, d, f) is right-handed
    fx = (W / 2.0) / np.tan(np.radians(hfov_deg) / 2.0)
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    uu, vv = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    dirs = ((vv - cx) / fx)[..., None] * r + ((uu - cy) / fx)[..., None] * d + f
    dirs = (dirs / np.linalg.norm(dirs, axis=-1, keepdims=True)).reshape(-1, 3)
    origin = np.array([0.0, 0.0, cam_height])
    surf = _Surfaces(origin, dirs)

    dominant = [np.array([0.0, 0.0, 1.0]), np.array([-1.0, 0.0, 0.0]), np.array([0.0, -1.0, 0.0])]
    groups: dict[int, int] = {}
    groups[surf.axis_plane(2, 0.0, [0, 0, 1], [(0, -50, wall), (1, -50, wall)])] = 0      # floor
    groups[surf.axis_plane(0, wall, [-1, 0, 0], [(1, -50, wall), (2, 0, 3.0)])] = 1       # wall x = 3
    groups[surf.axis_plane(1, wall, [0, -1, 0], [(0, -50, wall), (2, 0, 3.0)])] = 2       # wall y = 3

    def visible(x, y):
        p = np.array([x, y, 0.0]) - origin
        z = p @ f
        if z <= 0:
            return False
        px = (p @ r) / z * fx + cx
        py = (p @ d) / z * fx + cy
        return 0.05 * W < px < 0.95 * W and 0.05 * H < py < 0.95 * H

    boxes = []
    tries = 0
    while len(boxes) < n_boxes and tries < 10000:
        tries += 1
        sx, sy, sz = rng.uniform(0.2, 0.6, 3)
        x, y = rng.uniform(0.5, wall - 0.4, 2)
        if x + sx / 2 > wall - 0.05 or y + sy / 2 > wall - 0.05 or not visible(x, y):
            continue
        boxes.append(((x - sx / 2, y - sy / 2, 0.0), (x + sx / 2, y + sy / 2, sz)))
    for lo, hi in boxes:
        for sid in surf.box(lo, hi):
            nrm = surf.normals[sid]
            for g, dn in enumerate(dominant):
                if np.allclose(nrm, dn):
                    groups[sid] = g

    if ramp:
        # A 1.2 m x 0.8 m ramp rising at 15 degrees away from the camera, resting on the floor.
        ang = np.radians(15.0)
        horiz = np.array([np.cos(yaw), np.sin(yaw), 0.0])
        a_dir = np.cos(ang) * horiz + np.array([0, 0, np.sin(ang)])
        b_dir = np.array([-np.sin(yaw), np.cos(yaw), 0.0])
        nrm = np.cross(a_dir, b_dir)
        nrm = nrm if nrm[2] > 0 else -nrm
        for _ in range(1000):
            s0 = rng.uniform(1.2, 2.0)
            if visible(*(s0 * horiz[:2])) and visible(*((s0 + 1.2) * horiz[:2])):
                break
        sid = surf.rect(np.array([s0 * horiz[0], s0 * horiz[1], 0.002]), a_dir, b_dir, 1.2, 0.8, nrm)
        dominant.append(nrm)
        groups[sid] = len(dominant) - 1

    pts, sid = _finish(surf, rng, H, W, noise_sigma, outlier_frac, outlier_range, nan_frac, None)
    S = len(surf.normals)
    sgroup = np.array([groups.get(s, -1) for s in range(S)], np.int32)
    prm = dict(DEPTH_PARAMS)
    if params:
        prm.update(params)
    return Frame(points=pts, dominant_normals=np.array(dominant, np.float32), params=prm, surface_id=sid,
                 surface_normals=np.array(surf.normals), surface_group=sgroup,
                 name=f"depth{H}x{W}", meta=dict(seed=seed, n_boxes=len(boxes), ramp=ramp))


# ----------------------------------------------------------------------------- spinning LiDAR

LIDAR_PARAMS = dict(lap_iters=3, lap_lambda=1.0, lap_kernel=3, bil_iters=2, bil_sigma_len=0.1, bil_sigma_ang=0.15,
                    bil_kernel=3, max_edge=0.5, min_dot=0.95, max_offset=0.0, min_triangles=0)


def lidar_scene(H: int = 64, W: int = 1024, seed: int = 103, n_cars: int = 20, range_noise: float = 0.02,
                missing_frac: float = 0.10, max_range: float = 100.0, elev_top_deg: float = 3.0,
                elev_bottom_deg: float = -25.0, sensor_height: float = 1.8, road_half: float = 4.0,
                curb: float = 0.15, facade: float = 10.0, facade_height: float = 15.0,
                params: dict | None = None) -> Frame:
    rng = np.random.default_rng(seed)
    elev = np.radians(np.linspace(elev_top_deg, elev_bottom_deg, H))          # row 0 = top
    azim = np.pi - np.arange(W) * (2 * np.pi / W)                             # decreasing: columns run right
    el, az = np.meshgrid(elev, azim, indexing="ij")
    dirs = np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], -1).reshape(-1, 3)
    surf = _Surfaces(np.array([0.0, 0.0, sensor_height]), dirs)
    far = 1e4
    groups: dict[int, int] = {}
    groups[surf.axis_plane(2, 0.0, [0, 0, 1], [(0, -far, far), (1, -road_half, road_half)])] = 0      # road
    for side in (+1, -1):
        y0, y1 = sorted((side * road_half, side * facade))
        groups[surf.axis_plane(2, curb, [0, 0, 1], [(0, -far, far), (1, y0, y1)])] = 0                 # sidewalk
        surf.axis_plane(1, side * road_half, [0, -side, 0], [(0, -far, far), (2, 0, curb)])            # curb face
        sid = surf.axis_plane(1, side * facade, [0, -side, 0], [(0, -far, far), (2, 0, facade_height)])
        if side == +1:
            groups[sid] = 1                                                                            # facade
    for _ in range(n_cars):
        while True:
            x = rng.uniform(-60, 60)
            if abs(x) > 6:
                break
        y = rng.uniform(-road_half + 1.0, road_half - 1.0)
        lo = (x - 2.25, y - 0.9, 0.0)
        hi = (x + 2.25, y + 0.9, 1.5)
        for sid in surf.box(lo, hi):
            if np.allclose(surf.normals[sid], [0, 0, 1]):
                groups[sid] = 0
            elif np.allclose(surf.normals[sid], [0, -1, 0]):
                groups[sid] = 1
    pts, sid = _finish(surf, rng, H, W, range_noise, 0.0, 0.0, missing_frac, max_range)
    S = len(surf.normals)
    sgroup = np.array([groups.get(s, -1) for s in range(S)], np.int32)
    prm = dict(LIDAR_PARAMS)
    if params:
        prm.update(params)
    dominant = np.array([[0, 0, 1], [0, -1, 0]], np.float32)
    return Frame(points=pts, dominant_normals=dominant, params=prm, surface_id=sid,
                 surface_normals=np.array(surf.normals), surface_group=sgroup,
                 name=f"lidar{H}x{W}", meta=dict(seed=seed, n_cars=n_cars))


# ----------------------------------------------------------------------------- named workloads


def rgbd_120x160(seed: int = 101) -> Frame:
    """Depth camera 120x160, 4 boxes, 5 mm noise, 2% NaN, K = 3."""
    return depth_camera_scene(120, 160, seed=seed, n_boxes=4, ramp=False, noise_sigma=0.005, nan_frac=0.02)


def rgbd_480x640(seed: int = 102) -> Frame:
    """Depth camera 480x640, 12 boxes + 15-degree ramp, 5 mm noise + 1% outliers (+/-0.3 m), 3% NaN, K = 4."""
    return depth_camera_scene(480, 640, seed=seed, n_boxes=12, ramp=True, noise_sigma=0.005, outlier_frac=0.01,
                              outlier_range=0.3, nan_frac=0.03)


def lidar_64x1024(seed: int = 103) -> Frame:
    """Spinning LiDAR 64x1024, 20 cars, 2 cm noise, 10% missing, K = 2."""
    return lidar_scene(64, 1024, seed=seed)


WORKLOADS = {
    "rgbd_120x160": rgbd_120x160,
    "rgbd_480x640": rgbd_480x640,
    "lidar_64x1024": lidar_64x1024,
}

MIXED_SIZES = [(120, 160), (240, 320), (480, 640), (64, 1024), (128, 2048)]


def mixed_frame(H: int, W: int, seed: int) -> Frame:
    """One frame of the mixed-size batch: depth sizes from the depth generator, LiDAR sizes from the LiDAR one."""
    if (H, W) in ((64, 1024), (128, 2048)):
        return lidar_scene(H, W, seed=seed)
    big = H * W >= 480 * 640
    return depth_camera_scene(H, W, seed=seed, n_boxes=12 if big else 4, ramp=big, noise_sigma=0.005,
                              outlier_frac=0.01 if big else 0.0, nan_frac=0.03 if big else 0.02)


def mixed_batch(n: int = 256, seed: int = 104) -> list[Frame]:
    """n frames with sizes drawn uniformly from MIXED_SIZES (one seed per frame derived from `seed`)."""
    rng = np.random.default_rng(seed)
    picks = rng.integers(0, len(MIXED_SIZES), n)
    return [mixed_frame(*MIXED_SIZES[int(k)], seed=seed * 1000 + i) for i, k in enumerate(picks)]

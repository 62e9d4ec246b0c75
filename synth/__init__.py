"""Seeded synthetic workloads shared by the tests, the smoke check and the benchmark (inputs only)."""
from .scenes import (Frame, depth_camera_scene, lidar_scene, rgbd_120x160, rgbd_480x640, lidar_64x1024,
                     mixed_frame, mixed_batch, WORKLOADS, MIXED_SIZES, DEPTH_PARAMS, LIDAR_PARAMS)

__all__ = ["Frame", "depth_camera_scene", "lidar_scene", "rgbd_120x160", "rgbd_480x640", "lidar_64x1024",
           "mixed_frame", "mixed_batch", "WORKLOADS", "MIXED_SIZES", "DEPTH_PARAMS", "LIDAR_PARAMS"]

"""Host-side arithmetic of the benchmark (no GPU): the algorithmic work per frame that the
roofline divides by, the FP32 peak it compares with, the whole-job throughput, and the rule that
keeps a recorded ncu traffic figure only while the kernel sources it was taken from are
unchanged."""
import os
import shutil

import pytest

import bench


def test_algorithmic_bytes_by_hand():
    # 12 B per point read; per triangle 12 B of normal, 1 B of mask, 4 B of label written
    H, W = 480, 640
    tri = 2 * (H - 1) * (W - 1)
    assert tri == 612162
    assert bench.algorithmic_bytes(H, W) == 12 * H * W + 17 * tri == 14093154


def test_algorithmic_flop_by_hand():
    H, W, K = 120, 160, 3
    prm = dict(lap_iters=5, lap_kernel=3, bil_iters=3, bil_kernel=3)
    f = bench.algorithmic_flop(H, W, prm, K)
    npx, tri = H * W, 2 * (H - 1) * (W - 1)
    lap = 16 * 8 * npx * 5                     # 8 window neighbours of a 3 x 3 kernel
    bil = 26 * 18 * tri * 3 + 30 * tri         # 18 window triangles of a 3 x 3 quad window
    cls = 5 * K * tri
    assert f["laplacian"] == lap
    assert f["bilateral"] == bil + cls
    assert f["total"] == lap + bil + cls
    # a 5 x 5 kernel has 24 neighbours and 50 window triangles
    f5 = bench.algorithmic_flop(H, W, dict(prm, lap_kernel=5, bil_kernel=5), K)
    assert f5["laplacian"] == 16 * 24 * npx * 5
    assert f5["bilateral"] == 26 * 50 * tri * 3 + 30 * tri + cls


def test_fp32_peak_and_throughput():
    assert bench.fp32_peak_tflops(152, 2070.0) == pytest.approx(80.54784)
    # two ranks of 612,162 triangles, the slower at 0.1 ms per step
    assert bench.aggregate_mtri_s(612162, 2, 0.1) == pytest.approx(2 * 612162 / 1e-4 / 1e6)


def _fake_tree(tmp_path, traffic, digest):
    """A copy of the kernel sources and one profile summary under tmp_path."""
    src = os.path.join(bench.ROOT, "paper_2007_12065_gb300", "csrc")
    dst = tmp_path / "paper_2007_12065_gb300" / "csrc"
    dst.mkdir(parents=True)
    for name in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, name), dst / name)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "frame_kernel_demo.md").write_text(
        "# summary\n\n    traffic_bytes_per_launch: %s\n    kernel_sources_sha256: %s\n" % (traffic, digest))
    return dst


def test_recorded_traffic_follows_the_kernel_sources(tmp_path, monkeypatch):
    digest = bench.kernel_source_hash()
    dst = _fake_tree(tmp_path, 1234567, digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_source_hash() == digest
    assert bench.recorded_traffic("frame_kernel", "demo") == 1234567.0
    assert bench.recorded_traffic("frame_kernel", "absent") is None
    # any edit of a kernel source drops the figure
    with open(dst / bench.KERNEL_SOURCES[0], "a") as f:
        f.write("\n// edited\n")
    assert bench.kernel_source_hash() != digest
    assert bench.recorded_traffic("frame_kernel", "demo") is None


def test_committed_profile_carries_a_traffic_figure():
    text = open(os.path.join(bench.ROOT, "profiles", "frame_kernel_rgbd_480x640.md")).read()
    keys = [line.split(":")[0].strip() for line in text.splitlines() if ":" in line]
    assert "traffic_bytes_per_launch" in keys and "kernel_sources_sha256" in keys


def test_one_iteration_work_by_hand():
    # a 480 x 640 frame: 307,200 points, 612,162 triangles
    px, tri = 480 * 640, 612162
    b, f = bench.one_iteration_work("laplacian", px, tri)
    assert b == 24 * 307200 == 7372800 and f == 128 * 307200
    b, f = bench.one_iteration_work("bilateral", px, tri)
    assert b == 24 * 307200 + 18 * 612162 and f == 468 * 612162
    b, f = bench.one_iteration_work("bilateral_iteration", px, tri)
    assert b == 36 * 612162 and f == 468 * 612162
    with pytest.raises(ValueError):
        bench.one_iteration_work("merge", px, tri)

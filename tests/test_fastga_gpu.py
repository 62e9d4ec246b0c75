"""Gaussian accumulator on the device (Section 6.1, Algorithm 3) against the oracle's brute-force
nearest cell, and dominant normals of the synthetic scenes recovered by it (Section 6.3)."""
import os

import numpy as np
import pytest

import oracle
from oracle import fastga
import synth

pytestmark = pytest.mark.gpu

TIE = 1e-6   # FP32 dot products of unit vectors: a different cell only on a near tie


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


def _device(env, normals, level, mask=None, stride=1):
    pl3d, ctx, torch = env
    n = len(normals)
    nd = torch.from_numpy(np.ascontiguousarray(normals, np.float32)).cuda()
    md = torch.from_numpy(np.ascontiguousarray(mask, np.uint8)).cuda() if mask is not None else None
    counts = torch.empty(20 * 4 ** level, dtype=torch.int32, device="cuda")
    cells = torch.empty(n, dtype=torch.int32, device="cuda")
    pl3d.pl3d_fastga(ctx, nd, md, n, level, stride, counts, cells)
    torch.cuda.synchronize()
    return counts.cpu().numpy(), cells.cpu().numpy()


def _compare(normals, level, dev_cells, ref_cells):
    """Every cell choice equals the oracle's, or lies within TIE of the best dot product."""
    V, F = fastga.icosahedron(level)
    N = fastga.cell_normals(V, F)
    sel = ref_cells >= 0
    assert np.array_equal(dev_cells >= 0, sel)
    x = np.asarray(normals, np.float64)[sel]
    x /= np.linalg.norm(x, axis=1)[:, None]
    d_dev = np.einsum("ij,ij->i", x, N[dev_cells[sel]])
    d_ref = np.einsum("ij,ij->i", x, N[ref_cells[sel]])
    diff = dev_cells[sel] != ref_cells[sel]
    assert np.all(d_ref - d_dev <= TIE), float((d_ref - d_dev).max())
    return int(diff.sum())


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_random_normals_find_the_nearest_cell(env, level):
    rng = np.random.default_rng(level)
    n = 200_000 if level <= 4 else 20_000
    x = rng.normal(size=(n, 3))
    x = (x / np.linalg.norm(x, axis=1)[:, None]).astype(np.float32)
    counts, cells = _device(env, x, level)
    ref_counts, ref_cells = fastga.accumulate(x, level)
    ties = _compare(x, level, cells, ref_cells)
    print(f"level {level}: {ties} near-tie choices of {n}")
    assert counts.sum() == n
    assert np.array_equal(counts, np.bincount(cells, minlength=len(counts)))


def test_frame_normals_mask_and_sampling(env):
    """The oracle's filtered normals of the 480x640 frame (FP32), with its mask and every third
    triangle sampled: same cells as the oracle up to near ties, same histogram otherwise."""
    f = synth.rgbd_480x640()
    op = oracle.OracleParams(**f.params)
    ref = oracle.extract_planes(f.points, op, f.dominant_normals, sensitivity=False)
    normals = ref["normals"].astype(np.float32)
    mask = ref["mask"].astype(np.uint8)
    counts, cells = _device(env, normals, 4, mask, stride=3)
    ref_counts, ref_cells = fastga.accumulate(normals, 4, mask, stride=3)
    ties = _compare(normals, 4, cells, ref_cells)
    print("frame near ties:", ties)
    moved = np.abs(counts.astype(np.int64) - ref_counts).sum()
    assert moved <= 2 * ties


def test_dominant_normals_of_the_scenes_are_recovered(env):
    """Section 6.3 end to end on the device: filtered normals of pl3d_extract_planes -> histogram
    -> peaks. Every dominant normal of the scene comes back within 3 degrees."""
    pl3d, ctx, torch = env
    for f in (synth.rgbd_480x640(), synth.lidar_64x1024()):
        H, W = f.points.shape[:2]
        n = 2 * (H - 1) * (W - 1)
        pts = torch.from_numpy(f.points).cuda()
        m = torch.empty(n, dtype=torch.uint8, device="cuda")
        nr = torch.empty((n, 3), device="cuda")
        lb = torch.empty(n, dtype=torch.int32, device="cuda")
        pl3d.pl3d_extract_planes(ctx, pts, H, W, pl3d.make_params(**f.params), np.array([[0, 0, 1]], np.float32), 1,
                                 m, nr, lb)
        counts = torch.empty(5120, dtype=torch.int32, device="cuda")
        pl3d.pl3d_fastga(ctx, nr, m, n, 4, 1, counts)
        c = counts.cpu().numpy()
        peaks, weights = pl3d.pl3d_fastga_peaks(4, c, v_min=0.002 * c.sum(), d_peak=0.2, max_peaks=8)
        for d in f.dominant_normals:
            d = d / np.linalg.norm(d)
            ang = np.degrees(np.arccos(np.clip(peaks @ d, -1, 1))).min()
            print(f.name, d.round(3), f"{ang:.2f} deg")
            assert ang < 3.0

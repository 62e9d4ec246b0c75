"""Pins of the FastGA oracle (Section 6) against the paper's printed table, closed forms and an
independent nearest-neighbour library."""
import json
import os

import numpy as np
import pytest

from oracle import fastga

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_icosahedron.json")))


def _edge_adjacent_angles(N, F):
    edges = {}
    for t, f in enumerate(F):
        for e in range(3):
            a, b = int(f[e]), int(f[(e + 1) % 3])
            edges.setdefault((min(a, b), max(a, b)), []).append(t)
    pairs = [v for v in edges.values()]
    assert all(len(v) == 2 for v in pairs)             # a closed two-manifold
    return np.degrees([np.arccos(np.clip(N[a] @ N[b], -1.0, 1.0)) for a, b in pairs])


@pytest.mark.parametrize("row", GOLDEN["levels"], ids=lambda r: f"level{r['level']}")
def test_paper_refinement_table(row):
    """Vertex and triangle counts of the table, and its separation: the smallest angle between the
    surface normals of two cells sharing an edge, to the table's 0.1 degree."""
    V, F = fastga.icosahedron(row["level"])
    assert len(V) == row["vertices"] and len(F) == row["triangles"]
    ang = _edge_adjacent_angles(fastga.cell_normals(V, F), F)
    assert round(float(ang.min()), 1) == row["separation_deg"]
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0)


@pytest.mark.parametrize("level", [1, 2, 3])
def test_neighbour_counts(level):
    """12 neighbours in the 1-ring vertex adjacency, 11 for the 60 cells that touch one of the 12
    five-valent vertices (the paper's 'maximum of 60')."""
    V, F = fastga.icosahedron(level)
    cnt = np.bincount([len(x) for x in fastga.neighbours(F)])
    assert cnt[11] == GOLDEN["cells_with_11_neighbours_at_most"] and cnt[12] == len(F) - 60
    assert cnt.sum() == len(F)


def _solid_angle(a, b, c):
    """Solid angle of the spherical triangle (a, b, c) (Van Oosterom and Strackee, 1983)."""
    num = np.einsum("ij,ij->i", a, np.cross(b, c))
    den = 1 + np.einsum("ij,ij->i", a, b) + np.einsum("ij,ij->i", b, c) + np.einsum("ij,ij->i", c, a)
    return 2 * np.arctan2(num, den)


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_cells_tile_the_sphere_and_children_tile_their_parent(level):
    """Outward, counter-clockwise cells covering 4 pi exactly; the four children of face p are
    faces 4p .. 4p+3 of the next level and cover exactly its spherical triangle."""
    V, F = fastga.icosahedron(level)
    om = _solid_angle(V[F[:, 0]], V[F[:, 1]], V[F[:, 2]])
    assert np.all(om > 0)
    assert abs(om.sum() - 4 * np.pi) < 1e-9
    V2, F2 = fastga.icosahedron(level + 1)
    assert np.allclose(V2[:len(V)], V)                  # refinement keeps the old vertices first
    om2 = _solid_angle(V2[F2[:, 0]], V2[F2[:, 1]], V2[F2[:, 2]])
    assert np.allclose(om2.reshape(-1, 4).sum(1), om, atol=1e-12)
    # child 1 keeps vertex b of its parent, child 0 vertex a, child 2 vertex c
    assert np.array_equal(F2[0::4, 0], F[:, 0]) and np.array_equal(F2[1::4, 1], F[:, 1])
    assert np.array_equal(F2[2::4, 2], F[:, 2])


def test_nearest_cell_matches_a_kd_tree():
    """Largest dot product = smallest Euclidean distance between unit vectors: scipy's KD tree
    over the cell normals must agree."""
    spatial = pytest.importorskip("scipy.spatial")
    V, F = fastga.icosahedron(3)
    N = fastga.cell_normals(V, F)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(20000, 3))
    x /= np.linalg.norm(x, axis=1)[:, None]
    _, kd = spatial.cKDTree(N).query(x)
    assert np.array_equal(fastga.nearest_cell(x, N), kd)


def test_accumulate_counts_sampling_and_mask():
    rng = np.random.default_rng(5)
    n = rng.normal(size=(1000, 3)).astype(np.float32)
    n /= np.linalg.norm(n, axis=1)[:, None]
    n[::7] = np.nan
    mask = (rng.random(1000) < 0.8).astype(np.uint8)
    counts, cells = fastga.accumulate(n, 2, mask, stride=3)
    expect = [i for i in range(0, 1000, 3) if mask[i] and np.isfinite(n[i]).all()]
    assert counts.sum() == len(expect) and len(counts) == 320
    assert np.array_equal(np.nonzero(cells >= 0)[0], expect)


def test_peaks_find_planted_directions_and_merge_close_ones():
    """Three planted directions (floor, two walls) come back as the three peaks; two directions
    2 degrees apart merge into their weighted mean when d_peak exceeds their distance."""
    level = 3
    V, F = fastga.icosahedron(level)
    N = fastga.cell_normals(V, F)
    dirs = np.array([[0.03, 0.05, 1], [1, 0.07, -0.04], [0.1, 1, 0.2]], float)
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    counts = np.zeros(len(F), np.int64)
    for d, w in zip(dirs, (900, 500, 300)):                      # bumps about 6 degrees wide
        counts += np.round(w * np.exp(-(1 - N @ d) / 5e-3)).astype(np.int64)
    pk, wt = fastga.peaks(counts, level, v_min=20, d_peak=0.1)
    assert len(pk) == 3 and list(wt) == sorted(wt, reverse=True)
    for p, d in zip(pk, dirs):
        assert np.degrees(np.arccos(np.clip(p @ d, -1, 1))) < 3.2   # within one cell separation
    # two isolated peaks 20 degrees apart (not 1-ring neighbours): distance 2 sin 10 deg = 0.347
    t = np.radians(20.0)
    a, b = np.array([0.02, 0.03, 1.0]), np.array([np.sin(t), 0.03, np.cos(t)])
    ca, cb = fastga.nearest_cell(np.stack([a, b]) / np.linalg.norm([a, b], axis=1)[:, None], N)
    assert cb not in fastga.neighbours(F)[ca]
    c2 = np.zeros(len(F), np.int64)
    c2[ca], c2[cb] = 300, 100
    pk2, wt2 = fastga.peaks(c2, level, v_min=10, d_peak=0.4)
    assert len(pk2) == 1 and wt2[0] == 400
    mean = 300 * N[ca] + 100 * N[cb]
    assert np.allclose(pk2[0], mean / np.linalg.norm(mean))
    pk3, wt3 = fastga.peaks(c2, level, v_min=10, d_peak=0.3)
    assert len(pk3) == 2 and list(wt3) == [300, 100]


def test_peak_plateau_and_threshold_by_hand():
    """The peak rule as defined: a plateau of two neighbouring cells gives one peak, at its lower
    index; a count equal to v_min is not above it."""
    level = 2
    V, F = fastga.icosahedron(level)
    N = fastga.cell_normals(V, F)
    nb = fastga.neighbours(F)
    a = 37
    b = max(nb[a])                      # a 1-ring neighbour with a higher index
    counts = np.zeros(len(F), np.int64)
    counts[a] = counts[b] = 50
    pk, wt = fastga.peaks(counts, level, v_min=10, d_peak=0.01)
    assert len(pk) == 1 and list(wt) == [50] and np.allclose(pk[0], N[a])
    lone = np.zeros(len(F), np.int64)
    lone[a] = 20
    assert len(fastga.peaks(lone, level, v_min=20, d_peak=0.01)[0]) == 0
    pk, wt = fastga.peaks(lone, level, v_min=19, d_peak=0.01)
    assert len(pk) == 1 and list(wt) == [20] and np.allclose(pk[0], N[a])

"""Pins for the FP64 oracle: facts the paper and the mathematics fix, not the oracle's own formulas.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign, a
transposed operand, an off-by-one window) fails at least one of them:

* mesh counts printed in the paper (golden) and vertex valences of the right-cut mesh;
* Algorithm 1/2 explicit arrays against the vertex lists (twins share an edge, reversed);
* region growing against an independent union-find over the explicit half-edges;
* Laplacian: zero motion on affine grids, convexity (no out-of-plane motion), hand cases;
* normals: the closed form A x B on affine grids, sensor-facing orientation;
* bilateral: fixed point, the box-filter limit (convolution), the identity limit, a
  two-triangle closed form, sharp creases preserved;
* group assignment: thresholds probed from both sides, ties, masks;
* whole path: noise-free scenes map to their ground-truth groups.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def affine_grid(H, W, o=(0.25, -0.5, 2.0), A=(0.0, 0.0625, 0.0), B=(0.0625, 0.0, 0.0)):
    """p(u, v) = o + u A + v B with dyadic numbers: exactly representable in FP32."""
    u, v = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    P = np.asarray(o)[None, None, :] + u[..., None] * np.asarray(A) + v[..., None] * np.asarray(B)
    return P.astype(np.float32)


def plane_grid(H, W, normal, dist, f=50.0, rng=None, nan_frac=0.0):
    """Pinhole rays (x right, y down, z forward) cut by the plane n . p = dist."""
    n = np.asarray(normal, np.float64)
    n = n / np.linalg.norm(n)
    u, v = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    d = np.stack([(v - (W - 1) / 2) / f, (u - (H - 1) / 2) / f, np.ones_like(u)], -1)
    t = dist / (d @ n)
    P = (t[..., None] * d).astype(np.float32)
    if rng is not None and nan_frac > 0:
        P[rng.random((H, W)) < nan_frac] = np.nan
    return P, n


# ----------------------------------------------------------------------------- mesh counts


def test_paper_triangle_counts():
    """Full grids keep 2(M-1)(N-1) triangles: the paper's 498,002 and 50,218."""
    cases = json.load(open(os.path.join(GOLDEN, "paper_triangle_counts.json")))["cases"]
    for c in cases:
        P = oracle.widen(affine_grid(c["rows"], c["cols"]))
        m, _ = oracle.mask(P, P, 0.0)
        assert int(m.sum()) == c["triangles"]
        T, Tmap = oracle.extract_triangles(P)
        assert T.shape[0] == c["triangles"]


@pytest.mark.parametrize("pos,lost", [((3, 4), 6), ((0, 0), 2), ((0, 6), 1), ((5, 6), 2), ((5, 0), 1),
                                      ((0, 3), 3), ((5, 3), 3), ((2, 0), 3), ((2, 6), 3)])
def test_vertex_valence_of_right_cut_mesh(pos, lost):
    """A NaN point removes exactly the triangles around it: 6 inside, 3 on an edge, 2 or 1 at corners
    (the diagonal runs from (u, v) to (u+1, v+1), so corners (0,0) and (M-1,N-1) touch two triangles)."""
    H, W = 6, 7
    P = affine_grid(H, W)
    P[pos] = np.nan
    m, _ = oracle.mask(oracle.widen(P), oracle.widen(P), 0.0)
    assert int(m.sum()) == 2 * (H - 1) * (W - 1) - lost


def test_edge_length_rule_strict():
    """Algorithm 4 rejects only when the longest edge is strictly greater than l_max."""
    P = affine_grid(4, 5, A=(0.0, 0.0625, 0.0), B=(0.0625, 0.0, 0.0))
    W = oracle.widen(P)
    diag = np.hypot(0.0625, 0.0625)
    m, e = oracle.mask(W, W, diag)
    assert m.all()
    assert np.allclose(e, diag, rtol=0, atol=1e-15)
    m, _ = oracle.mask(W, W, np.nextafter(diag, 0))
    assert not m.any()
    m, _ = oracle.mask(W, W, 0.0)   # disabled
    assert m.all()


# ----------------------------------------------------------------------------- Algorithms 1 and 2


@pytest.mark.parametrize("seed", range(6))
def test_halfedges_are_reversed_shared_edges(seed):
    """Every twin pair of Algorithm 2 joins two triangles of Algorithm 1 along the same edge, reversed;
    HE is an involution; and the twins are exactly the implicit neighbour rule."""
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(2, 9)), int(rng.integers(2, 9))
    P = affine_grid(H, W)
    P[rng.random((H, W)) < 0.2] = np.nan
    T, Tmap = oracle.extract_triangles(oracle.widen(P))
    HE = oracle.extract_halfedges(Tmap, H, W, T.shape[0])
    # every edge shared by two valid triangles, found by brute force over vertex pairs
    edges = {}
    for t in range(T.shape[0]):
        for e in range(3):
            a, b = int(T[t, e]), int(T[t, (e + 1) % 3])
            edges[(a, b)] = 3 * t + e
    for h in range(HE.shape[0]):
        t, e = divmod(h, 3)
        a, b = int(T[t, e]), int(T[t, (e + 1) % 3])
        twin = edges.get((b, a), -1)
        assert HE[h] == twin, (h, HE[h], twin)
        if HE[h] >= 0:
            assert HE[HE[h]] == h
    # implicit rule == explicit twins (GID space)
    inv = {int(i): g for g, i in enumerate(Tmap) if i >= 0}
    for h in range(HE.shape[0]):
        if HE[h] < 0:
            continue
        g1, g2 = inv[h // 3], inv[int(HE[h]) // 3]
        assert g2 in oracle.triangle_twins(g1, H, W)


@pytest.mark.parametrize("seed", range(4))
def test_extracted_triangles_are_exactly_the_valid_ones(seed):
    """Algorithm 1 keeps a triangle iff its three vertices are valid: |T| is 2 (H-1)(W-1) minus
    the triangles with a NaN corner, counted here over the quads' corners (first takes p1, p2,
    p3 and second p1, p3, p4); every T entry has three finite vertices; T_map inverts T."""
    rng = np.random.default_rng(40 + seed)
    H, W = int(rng.integers(2, 10)), int(rng.integers(2, 10))
    P = affine_grid(H, W)
    P[rng.random((H, W)) < 0.25] = np.nan
    bad = np.isnan(P[..., 0])
    want = 0
    for u in range(H - 1):
        for v in range(W - 1):
            p1, p2, p3, p4 = bad[u, v], bad[u, v + 1], bad[u + 1, v + 1], bad[u + 1, v]
            want += int(not (p1 or p2 or p3)) + int(not (p1 or p3 or p4))
    T, Tmap = oracle.extract_triangles(oracle.widen(P))
    assert T.shape[0] == want
    flat = P.reshape(-1, 3)
    assert np.isfinite(flat[T.reshape(-1), 0]).all()
    kept = np.nonzero(Tmap >= 0)[0]
    assert kept.size == want and np.array_equal(Tmap[kept], np.arange(want))


def test_any_non_finite_coordinate_makes_the_point_invalid():
    """Sections 3 and 4.2: a missing return leaves a non-finite point in the organized cloud, and
    such a point is invalid whichever coordinate is non-finite -- inf in x, -inf in z, NaN in y
    only or in z only. It widens to NaN in all three coordinates; Algorithm 1 keeps only the
    triangles whose three corners have all coordinates finite (counted over the quads' corners);
    the whole path gives the same outputs, bit for bit, as the frame with those points written
    all-NaN (so no filter reads a finite coordinate of an invalid point)."""
    f = synth.depth_camera_scene(12, 14, seed=77, n_boxes=1, nan_frac=0.0)
    pts = f.points.copy()
    hits = [((3, 4), 0, np.inf), ((5, 6), 1, np.nan), ((7, 8), 2, np.nan), ((8, 3), 2, -np.inf),
            ((0, 5), 0, -np.inf), ((6, 11), 1, np.inf)]
    for (u, v), c, val in hits:
        pts[u, v, c] = val
    ok = np.isfinite(pts).all(-1)
    assert (~ok).sum() == len(hits)
    wid = oracle.widen(pts)
    assert np.isnan(wid[~ok]).all()
    assert np.array_equal(wid[ok], pts[ok].astype(np.float64))
    bad = ~ok
    H, W = bad.shape
    want = sum(int(not (bad[u, v] or bad[u, v + 1] or bad[u + 1, v + 1])) +
               int(not (bad[u, v] or bad[u + 1, v + 1] or bad[u + 1, v]))
               for u in range(H - 1) for v in range(W - 1))
    T, _ = oracle.extract_triangles(wid)
    assert T.shape[0] == want
    all_nan = pts.copy()
    all_nan[bad] = np.nan
    p = oracle.OracleParams(**f.params)
    a = oracle.extract_planes(pts, p, f.dominant_normals, sensitivity=False)
    b = oracle.extract_planes(all_nan, p, f.dominant_normals, sensitivity=False)
    for k in ("smoothed", "normals", "mask", "groups", "labels"):
        assert np.array_equal(a[k], b[k], equal_nan=a[k].dtype.kind == "f"), k
    assert np.isnan(a["smoothed"][bad]).all()
    assert (a["mask"] == 1).sum() <= want


def test_edge_test_reads_smoothed_vertices_validity_reads_raw():
    """Algorithm 4 measures edges on the points after smoothing; Algorithm 1 takes validity from
    the raw cloud. A spike in one copy only moves the decision of the copy that is measured."""
    P = oracle.widen(affine_grid(4, 5, A=(0.0, 0.0625, 0.0), B=(0.0625, 0.0, 0.0)))
    spiked = P.copy()
    spiked[1, 2, 2] += 1.0
    m, _ = oracle.mask(spiked, P, 0.1)            # raw spike, smooth surface: all kept
    assert m.all()
    m, e = oracle.mask(P, spiked, 0.1)            # the smoothed copy carries the spike
    touching = ~(e <= 0.1)
    assert 0 < touching.sum() < m.size and not m[touching].any() and m[~touching].all()
    holed = P.copy()
    holed[1, 2] = np.nan
    m, _ = oracle.mask(holed, P, 0.1)             # validity from the raw copy
    assert (m == 0).sum() == 6                    # the six triangles around an interior vertex


def test_first_triangle_vertex_order_and_gid():
    """Algorithm 1: first = {p3, p2, p1}, second = {p1, p4, p3}; GID = 2 (u (N-1) + v) + k."""
    H, W = 3, 4
    T, Tmap = oracle.extract_triangles(oracle.widen(affine_grid(H, W)))
    u, v = 1, 2
    p1, p2, p3, p4 = u * W + v, u * W + v + 1, (u + 1) * W + v + 1, (u + 1) * W + v
    g = 2 * (u * (W - 1) + v)
    assert list(T[Tmap[g]]) == [p3, p2, p1]
    assert list(T[Tmap[g + 1]]) == [p1, p4, p3]


# ----------------------------------------------------------------------------- region growing


class _UF:
    def __init__(self, n):
        self.p = list(range(n))

    def find(self, x):
        while self.p[x] != x:
            self.p[x] = self.p[self.p[x]]
            x = self.p[x]
        return x

    def union(self, a, b):
        a, b = self.find(a), self.find(b)
        if a != b:
            self.p[max(a, b)] = min(a, b)


def brute_labels(P, G, tri_min=0, C=None, nd=None, max_offset=0.0):
    """Components over the explicit half-edges of Algorithms 1-2 with a textbook union-find."""
    H, W = P.shape[:2]
    T, Tmap = oracle.extract_triangles(oracle.widen(P))
    HE = oracle.extract_halfedges(Tmap, H, W, T.shape[0])
    inv = {int(i): g for g, i in enumerate(Tmap) if i >= 0}
    n = G.shape[0]
    uf = _UF(n)
    for h in range(HE.shape[0]):
        if HE[h] < 0:
            continue
        a, b = inv[h // 3], inv[int(HE[h]) // 3]
        if G[a] == 255 or G[a] != G[b]:
            continue
        if max_offset > 0 and abs(float(nd[G[a]] @ (C[a] - C[b]))) > max_offset:
            continue
        uf.union(a, b)
    lab = np.array([uf.find(i) if G[i] != 255 else -1 for i in range(n)], np.int64)
    if tri_min > 0:
        roots, counts = np.unique(lab[lab >= 0], return_counts=True)
        small = set(int(r) for r, c in zip(roots, counts) if c <= tri_min)
        lab = np.array([-1 if l in small else l for l in lab])
    return lab


@pytest.mark.parametrize("seed", range(12))
def test_labels_match_union_find_on_tiny_grids(seed):
    rng = np.random.default_rng(100 + seed)
    H, W = int(rng.integers(2, 9)), int(rng.integers(2, 9))
    P = affine_grid(H, W)
    P[rng.random((H, W)) < 0.15] = np.nan
    n = 2 * (H - 1) * (W - 1)
    m, _ = oracle.mask(oracle.widen(P), oracle.widen(P), 0.0)
    G = rng.integers(0, 3, n).astype(np.uint8)
    G[rng.random(n) < 0.2] = 255
    G[m == 0] = 255       # triangles with a NaN vertex have no group (Algorithm 4 runs on T only)
    tri_min = int(rng.integers(0, 4))
    got = oracle.label(G, H, W, tri_min=tri_min)
    want = brute_labels(P, G, tri_min)
    np.testing.assert_array_equal(got, want)


def test_labels_with_offset_test_match_union_find():
    rng = np.random.default_rng(7)
    H, W = 7, 8
    P = affine_grid(H, W)
    P[..., 2] += rng.normal(0, 0.01, (H, W)).astype(np.float32)
    Pw = oracle.widen(P)
    C, _ = oracle.triangle_geometry(Pw)
    nd = oracle.normalize_dominant(np.array([[0, 0, 1], [1, 0, 0]], np.float32))
    n = C.shape[0]
    G = np.zeros(n, np.uint8)
    G[rng.random(n) < 0.1] = 1
    got = oracle.label(G, H, W, C, nd, max_offset=0.006)
    want = brute_labels(P, G, 0, C, nd, 0.006)
    np.testing.assert_array_equal(got, want)


def test_labels_with_offset_test_on_a_tilted_plane():
    """The offset test along a dominant normal with three non-zero components, on a plane
    perpendicular to it with range noise along it: every component of the centroid difference
    counts."""
    rng = np.random.default_rng(11)
    H, W = 8, 9
    nrm = np.array([0.36, 0.48, 0.8])
    A = np.array([0.8, 0.0, -0.36])
    B = np.cross(nrm, A)
    u, v = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    P = (0.05 * u[..., None] * A + 0.05 * v[..., None] * B
         + rng.normal(0, 0.01, (H, W))[..., None] * nrm).astype(np.float32)
    C, _ = oracle.triangle_geometry(oracle.widen(P))
    nd = oracle.normalize_dominant(np.array([nrm, [1, 0, 0]], np.float32))
    n = C.shape[0]
    G = np.zeros(n, np.uint8)
    got = oracle.label(G, H, W, C, nd, max_offset=0.003)
    want = brute_labels(P, G, 0, C, nd, 0.003)
    np.testing.assert_array_equal(got, want)
    assert 1 < len(np.unique(got)) < n      # the threshold splits the plane, not every triangle


def test_uniform_plane_is_one_component():
    H, W = 9, 11
    n = 2 * (H - 1) * (W - 1)
    lab = oracle.label(np.zeros(n, np.uint8), H, W)
    assert (lab == 0).all()
    lab = oracle.label(np.zeros(n, np.uint8), H, W, tri_min=n)      # |T| > tri_min fails
    assert (lab == -1).all()
    lab = oracle.label(np.zeros(n, np.uint8), H, W, tri_min=n - 1)
    assert (lab == 0).all()


def test_label_is_min_gid_of_component():
    rng = np.random.default_rng(3)
    H, W = 8, 8
    n = 2 * (H - 1) * (W - 1)
    G = rng.integers(0, 2, n).astype(np.uint8)
    lab = oracle.label(G, H, W)
    for l in np.unique(lab):
        members = np.nonzero(lab == l)[0]
        assert members.min() == l


# ----------------------------------------------------------------------------- Laplacian (Eq. 1-2)


@pytest.mark.parametrize("kernel", [3, 5])
def test_laplacian_affine_grid_does_not_move(kernel):
    """Symmetric inverse-distance weights cancel on an affine grid (no NaN)."""
    P = oracle.widen(affine_grid(12, 13, A=(0.0, 0.0625, 0.125), B=(0.0625, 0.0, -0.03125)))
    S = oracle.laplacian(P, kernel, 1.0, 4)
    assert np.abs(S - P).max() < 1e-13


def test_laplacian_is_convex_no_out_of_plane_motion():
    """lambda in [0, 1] makes each update a convex combination, so no point leaves the plane."""
    rng = np.random.default_rng(5)
    P, n = plane_grid(20, 24, normal=(0.3, -0.4, -1.0), dist=-2.0, rng=rng, nan_frac=0.1)
    Pw = oracle.widen(P)
    d_in = np.nanmax(np.abs(Pw @ n + 2.0))
    for lam in (0.3, 1.0):
        S = oracle.laplacian(Pw, 3, lam, 5)
        d_out = np.nanmax(np.abs(S @ n + 2.0))
        assert d_out <= d_in + 1e-12
        np.testing.assert_array_equal(np.isnan(S), np.isnan(Pw))


def test_laplacian_lambda_zero_and_border_pinned():
    rng = np.random.default_rng(6)
    P = oracle.widen(rng.normal(0, 1, (9, 10, 3)).astype(np.float32))
    assert np.array_equal(oracle.laplacian(P, 3, 0.0, 3), P)
    for kernel in (3, 5):
        r = kernel // 2
        S = oracle.laplacian(P, kernel, 1.0, 3)
        border = np.ones((9, 10), bool)
        border[r:-r, r:-r] = False
        assert np.array_equal(S[border], P[border])
        assert not np.array_equal(S[~border], P[~border])


def test_laplacian_hand_cases():
    """3x3 grid, kernel 3: only the centre is filtered (border pinned)."""
    P = np.full((3, 3, 3), np.nan)
    P[1, 1] = (0, 0, 0)
    P[1, 2] = (1, 0, 0)          # distance 1 -> w = 1
    P[0, 1] = (0, 2, 0)          # distance 2 -> w = 1/2
    S = oracle.laplacian(P, 3, 1.0, 1)
    # (1 * (1,0,0) + 1/2 * (0,2,0)) / (1 + 1/2) = (2/3, 2/3, 0)
    np.testing.assert_allclose(S[1, 1], (2 / 3, 2 / 3, 0), atol=1e-15)
    S = oracle.laplacian(P, 3, 0.5, 1)
    np.testing.assert_allclose(S[1, 1], (1 / 3, 1 / 3, 0), atol=1e-15)
    # a neighbour at distance 0 carries no weight; alone it leaves the point where it is
    Q = np.full((3, 3, 3), np.nan)
    Q[1, 1] = (1, 2, 3)
    Q[2, 2] = (1, 2, 3)
    assert np.array_equal(oracle.laplacian(Q, 3, 1.0, 2)[1, 1], Q[1, 1])
    # an isolated point stays put; NaN stays NaN
    R = np.full((3, 3, 3), np.nan)
    R[1, 1] = (1, 2, 3)
    S = oracle.laplacian(R, 3, 1.0, 1)
    assert np.array_equal(S[1, 1], R[1, 1]) and np.isnan(S[0, 0]).all()


def test_laplacian_jacobi_two_iterations_by_hand():
    """A 1x5 interior row inside a 3x7 grid of NaN: Jacobi reads only the previous iterate."""
    P = np.full((3, 7, 3), np.nan)
    xs = [0.0, 1.0, 3.0, 4.0, 8.0]
    for i, x in enumerate(xs):
        P[1, 1 + i] = (x, 0, 0)
    lam = 0.5

    def step(row):
        # each interior point has its row neighbours v-1, v+1 (border columns and other rows are NaN)
        out = list(row)
        for i in range(len(row)):
            nb = [row[j] for j in (i - 1, i + 1) if 0 <= j < len(row)]
            w = [1 / abs(x - row[i]) for x in nb]
            out[i] = row[i] + lam * sum(wi * (x - row[i]) for wi, x in zip(w, nb)) / sum(w)
        return out
    r1 = step(xs)
    np.testing.assert_allclose(oracle.laplacian(P, 3, lam, 1)[1, 1:6, 0], r1, atol=1e-14)
    np.testing.assert_allclose(oracle.laplacian(P, 3, lam, 2)[1, 1:6, 0], step(r1), atol=1e-14)


def test_laplacian_two_interior_points_read_the_previous_iterate():
    """3x4 grid, kernel 3: the interior points A (1,1) and B (1,2) see each other; the border
    points C (1,0) and D (1,3) each sit in one window only. By hand, with lambda = 1:
    |B - A| = 5 (w = 1/5), |C - A| = 2 (w = 1/2), |D - B| = 12 (w = 1/12);
    A' = [(3,4,0)/5 + (0,-2,0)/2] / (7/10) = (6/7, -2/7, 0);
    B' = (3,4,0) + [(-3,-4,0)/5 + (0,0,12)/12] / (17/60) = (15/17, 20/17, 60/17).
    In 1-D the weighted differences are only signs, so this 2-D case is what separates Jacobi
    from an in-place (Gauss-Seidel) sweep, which would move B with A' instead of A."""
    P = np.full((3, 4, 3), np.nan)
    P[1, 1] = (0, 0, 0)
    P[1, 2] = (3, 4, 0)
    P[1, 0] = (0, -2, 0)
    P[1, 3] = (3, 4, 12)
    S = oracle.laplacian(P, 3, 1.0, 1)
    np.testing.assert_allclose(S[1, 1], (6 / 7, -2 / 7, 0), atol=1e-15)
    np.testing.assert_allclose(S[1, 2], (15 / 17, 20 / 17, 60 / 17), atol=1e-14)
    assert np.array_equal(S[1, 0], P[1, 0]) and np.array_equal(S[1, 3], P[1, 3])


def test_laplacian_equivariance():
    """Rigid motions commute with the filter; a sign slip in the update would still pass this, the
    hand cases above would not."""
    rng = np.random.default_rng(8)
    P = oracle.widen(rng.normal(0, 1, (8, 9, 3)).astype(np.float32))
    P[2, 3] = np.nan
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.linalg.det(q))
    t = np.array([1.0, -2.0, 0.5])
    S = oracle.laplacian(P, 3, 0.7, 3)
    S2 = oracle.laplacian(P @ q.T + t, 3, 0.7, 3)
    np.testing.assert_allclose(S2, S @ q.T + t, atol=1e-12)


# ----------------------------------------------------------------------------- normals (Section 5.2)


@pytest.mark.parametrize("A,B", [((0.0, 0.0625, 0.0), (0.0625, 0.0, 0.0)),
                                 ((0.0, 0.0625, 0.03125), (0.0625, 0.0, -0.125)),
                                 ((0.125, 0.0, 0.0), (0.0, 0.0, 0.0625))])
def test_normals_on_affine_grid_are_a_cross_b(A, B):
    """For p = o + u A + v B both triangles of every quad have normal A x B / |A x B|."""
    P = oracle.widen(affine_grid(5, 6, A=A, B=B))
    C, N = oracle.triangle_geometry(P)
    want = np.cross(A, B)
    want = want / np.linalg.norm(want)
    np.testing.assert_allclose(N, np.broadcast_to(want, N.shape), atol=1e-14)
    T, _ = oracle.extract_triangles(P)
    np.testing.assert_allclose(C, P.reshape(-1, 3)[T].mean(axis=1), atol=1e-14)


def test_fronto_parallel_normal_faces_sensor():
    """Optical frame (x right, y down, z forward): a wall in front of the camera has normal (0, 0, -1)."""
    P, _ = plane_grid(6, 8, normal=(0, 0, 1), dist=2.0)
    _, N = oracle.triangle_geometry(oracle.widen(P))
    np.testing.assert_allclose(N, np.broadcast_to([0, 0, -1.0], N.shape), atol=1e-6)


def test_tilted_plane_normals_face_sensor():
    rng = np.random.default_rng(9)
    for _ in range(5):
        n = rng.normal(size=3)
        n[2] = -abs(n[2]) - 0.5          # plane in front of the camera, facing it
        P, nu = plane_grid(7, 9, normal=n, dist=-2.0)
        Pw = oracle.widen(P)
        C, N = oracle.triangle_geometry(Pw)
        assert (np.einsum("ij,ij->i", N, C) < 0).all()   # facing the sensor at the origin
        np.testing.assert_allclose(np.abs(N @ nu), 1.0, atol=1e-5)


def test_degenerate_triangle_has_no_normal_but_keeps_its_centroid():
    """A triangle whose cross product is at most 1e-20 long has no normal (NaN), while its centroid
    stays. Grids scaled to 1e-11 (cross ~ 2e-24 ... 1e-22) and to 1e-9 (cross ~ 1e-18) sit on
    either side of the threshold."""
    for scale, none in ((1e-11, True), (1e-9, False)):
        P = oracle.widen(affine_grid(4, 5, o=(0.0, 0.0, 0.0), A=(0.0, 1.0, 0.0), B=(1.0, 0.0, 0.0))) * scale
        C, N = oracle.triangle_geometry(P)
        assert np.isfinite(C).all()
        assert np.isnan(N).all() if none else np.isfinite(N).all()


def test_nan_vertex_gives_nan_triangle():
    P = affine_grid(4, 4)
    P[1, 1, 2] = np.inf       # any non-finite coordinate invalidates the point
    C, N = oracle.triangle_geometry(oracle.widen(P))
    bad = np.isnan(N[:, 0])
    assert bad.sum() == 6 and np.isnan(C[bad]).all()


# ----------------------------------------------------------------------------- bilateral (Eq. 3-6)


def test_bilateral_constant_field_is_fixed_point():
    P = oracle.widen(affine_grid(9, 10, A=(0.0, 0.0625, 0.03125), B=(0.0625, 0.0, 0.0)))
    C, N = oracle.triangle_geometry(P)
    Nf = oracle.bilateral(C, N, 9, 10, 3, 0.1, 0.15, 4)
    np.testing.assert_allclose(Nf, N, atol=1e-14)


def _box_filter_normals(N, H, W, r, iters):
    """Unweighted window mean via summed shifted copies: the sigma -> infinity limit of Eq. 3."""
    Hq, Wq = H - 1, W - 1
    cur = N.reshape(Hq, Wq, 2, 3).copy()
    for _ in range(iters):
        valid = ~np.isnan(cur[..., 0])
        z = np.where(valid[..., None], cur, 0.0).sum(axis=2)           # both triangles of a quad
        pad = np.pad(z, ((r, r), (r, r), (0, 0)))
        s = sum(pad[r + du:r + du + Hq, r + dv:r + dv + Wq] for du in range(-r, r + 1) for dv in range(-r, r + 1))
        s = s / np.linalg.norm(s, axis=-1, keepdims=True)
        cur = np.where(valid[..., None], s[:, :, None, :], np.nan)
    return cur.reshape(-1, 3)


@pytest.mark.parametrize("kernel,iters", [(3, 1), (3, 2), (5, 1)])
def test_bilateral_large_sigma_is_box_mean(kernel, iters):
    rng = np.random.default_rng(10 + kernel)
    H, W = 8, 11
    P = oracle.widen(rng.normal(0, 1, (H, W, 3)).astype(np.float32))
    P[rng.random((H, W)) < 0.1] = np.nan
    C, N = oracle.triangle_geometry(P)
    got = oracle.bilateral(C, N, H, W, kernel, 1e9, 1e9, iters)
    want = _box_filter_normals(N, H, W, kernel // 2, iters)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want[:, 0])
    np.testing.assert_allclose(got[ok], want[ok], atol=1e-9)


def test_bilateral_tiny_sigma_is_identity():
    rng = np.random.default_rng(11)
    P = oracle.widen(rng.normal(0, 1, (7, 8, 3)).astype(np.float32))
    C, N = oracle.triangle_geometry(P)
    got = oracle.bilateral(C, N, 7, 8, 3, 1e-6, 1e-6, 3)
    np.testing.assert_allclose(got, N, rtol=0, atol=1e-15)   # self weight 1, every other weight underflows


def test_bilateral_two_triangles_closed_form():
    """A single quad: each triangle sees itself (weight 1) and its partner (weight w), so after one
    iteration n1' is n1 rotated towards n2 by atan(w sin t / (1 + w cos t))."""
    P = np.array([[[0, 0, 0], [1, 0, 0]], [[0, 1, 0.4], [1, 1, 0.0]]], np.float32)
    C, N = oracle.triangle_geometry(oracle.widen(P))
    sc, ss = 0.8, 0.6
    cosang = float(N[0] @ N[1])
    theta = np.arccos(cosang)
    w = np.exp(-np.sum((C[0] - C[1]) ** 2) / (2 * sc * sc)) * np.exp(-np.sum((N[0] - N[1]) ** 2) / (2 * ss * ss))
    Nf = oracle.bilateral(C, N, 2, 2, 3, sc, ss, 1)
    rot = np.arctan2(w * np.sin(theta), 1 + w * cosang)
    assert np.isclose(np.arccos(np.clip(Nf[0] @ N[0], -1, 1)), rot, atol=1e-7)
    assert np.isclose(np.arccos(np.clip(Nf[1] @ N[1], -1, 1)), rot, atol=1e-7)
    # the two rotate towards each other, in the plane they span
    assert Nf[0] @ N[1] > cosang and Nf[1] @ N[0] > cosang
    assert abs(np.linalg.det(np.stack([Nf[0], N[0], N[1]]))) < 1e-12


def test_bilateral_keeps_sharp_crease():
    """A 90-degree crease: W_s = exp(-2 / (2 sigma_s^2)) ~ 1e-19 keeps the two sides apart."""
    H, W = 10, 12
    u, v = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    x = v * 0.03125
    z = np.where(v <= 5, 1.0, 1.0 + (v - 5) * 0.03125)
    x = np.where(v <= 5, x, 5 * 0.03125)
    P = np.stack([x, u * 0.03125, z], -1).astype(np.float32)
    C, N = oracle.triangle_geometry(oracle.widen(P))
    Nf = oracle.bilateral(C, N, H, W, 3, 0.1, 0.15, 3)
    q = np.arange(N.shape[0]) // 2
    col = q % (W - 1)
    left, right = col < 5, col > 5
    np.testing.assert_allclose(Nf[left], N[left], atol=1e-6)
    np.testing.assert_allclose(Nf[right], N[right], atol=1e-6)
    assert abs(N[left][0] @ N[right][0]) < 1e-12


# ----------------------------------------------------------------------------- group assignment (Algorithm 4)


def test_classify_thresholds_ties_and_masks():
    nd = oracle.normalize_dominant(np.array([[0, 0, 2], [0, 0, 1], [1, 0, 0]], np.float32))
    ang = 0.95
    th = np.arccos(ang)
    d = 1e-7
    normals = np.array([
        [np.sin(th - d), 0, np.cos(th - d)],      # just inside -> group 0 (tie with group 1, first wins)
        [np.sin(th + d), 0, np.cos(th + d)],      # just outside -> 255
        [1, 0, 0],                                # group 2
        [-1, 0, 0],                               # opposite of group 2: signed dot -> 255
        [0, 0, 1],                                # masked out -> 255
        [np.nan, np.nan, np.nan],                 # no normal -> 255
        [np.cos(0.1), 0, np.sin(0.1)],            # closer to group 2 than 0
    ])
    m = np.array([1, 1, 1, 1, 0, 1, 1], np.uint8)
    G, best, second = oracle.classify(normals, m, nd, ang)
    assert list(G) == [0, 255, 2, 255, 255, 255, 2]
    assert best[0] == second[0]                   # the tie is visible to the near-threshold report
    # exactly at the threshold is kept (reject only when strictly below)
    G, _, _ = oracle.classify(np.array([[0.0, 0.6, 0.8]]), np.ones(1, np.uint8),
                              oracle.normalize_dominant(np.array([[0, 0, 1]], np.float32)), 0.8)
    assert G[0] == 0


def test_normalize_dominant_rejects_zero():
    with pytest.raises(ValueError):
        oracle.normalize_dominant(np.zeros((1, 3), np.float32))
    nd = oracle.normalize_dominant(np.array([[3, 4, 0]], np.float32))
    np.testing.assert_allclose(nd, [[0.6, 0.8, 0.0]])


# ----------------------------------------------------------------------------- whole path


@pytest.mark.parametrize("scene", ["depth", "lidar"])
def test_noise_free_scene_maps_to_ground_truth(scene):
    """On noise-free scenes, triangles well inside a ground-truth planar surface get that surface's group
    and every segment holds a single group."""
    if scene == "depth":
        f = synth.depth_camera_scene(60, 80, seed=1, n_boxes=3, ramp=True, noise_sigma=0.0, nan_frac=0.0)
    else:
        f = synth.lidar_scene(32, 512, seed=2, n_cars=8, range_noise=0.0, missing_frac=0.0)
    p = oracle.OracleParams(**f.params)
    r = oracle.extract_planes(f.points, p, f.dominant_normals)
    H, W = f.H, f.W
    sid = f.surface_id
    # surface id per quad when all four corners and their 2-ring agree (away from creases)
    from numpy.lib.stride_tricks import sliding_window_view
    pad = np.pad(sid, 3, constant_values=-2)
    win = sliding_window_view(pad, (8, 8))[:H - 1, :W - 1]
    same = (win == win[..., 3:4, 3:4]).all(axis=(-1, -2)) & (sid[:-1, :-1] >= 0)
    quad_sid = np.where(same, sid[:-1, :-1], -1)
    tri_sid = np.repeat(quad_sid.reshape(-1), 2)
    inside = (tri_sid >= 0) & (r["mask"] == 1)
    want = f.surface_group[tri_sid[inside]]
    got = r["groups"][inside].astype(np.int64)
    got[got == 255] = -1
    assert inside.sum() > 1000
    assert (got == want).mean() > 0.999
    lab = r["labels"]
    for l in np.unique(lab[lab >= 0]):
        assert len(np.unique(r["groups"][lab == l])) == 1


# ----------------------------------------------------------------------------- sensitivity instrumentation


def test_jitter_off_is_the_plain_filter():
    rng = np.random.default_rng(20)
    P = oracle.widen(rng.normal(0, 1, (9, 11, 3)).astype(np.float32))
    assert np.array_equal(oracle.laplacian(P, 3, 0.8, 3), oracle.laplacian(P, 3, 0.8, 3, eps=0.0, seed=99))
    C, N = oracle.triangle_geometry(P)
    assert np.array_equal(oracle.bilateral(C, N, 9, 11, 3, 0.5, 0.3, 2),
                          oracle.bilateral(C, N, 9, 11, 3, 0.5, 0.3, 2, eps=0.0, seed=5))


def test_jitter_moves_a_well_conditioned_frame_by_order_eps():
    """Every update scaled by (1 +- eps): on a smooth noisy plane the outputs move by O(eps) and the
    signs depend on the seed."""
    rng = np.random.default_rng(21)
    P, _ = plane_grid(24, 30, normal=(0.2, -0.3, -1.0), dist=-2.0)
    P = P + rng.normal(0, 0.002, P.shape).astype(np.float32)
    W_ = oracle.widen(P)
    eps = 2.0 ** -21
    S = oracle.laplacian(W_, 3, 1.0, 4)
    S1 = oracle.laplacian(W_, 3, 1.0, 4, eps, 1)
    S2 = oracle.laplacian(W_, 3, 1.0, 4, eps, 2)
    d1 = np.abs(S1 - S).max()
    assert 0 < d1 < 100 * eps * np.abs(S - W_).max()
    assert not np.array_equal(S1, S2)
    C, N = oracle.triangle_geometry(S)
    Nb = oracle.bilateral(C, N, 24, 30, 3, 0.1, 0.15, 3)
    Nj = oracle.bilateral(C, N, 24, 30, 3, 0.1, 0.15, 3, eps, 3)
    assert 0 < np.abs(Nj - Nb).max() < 100 * eps


def test_ill_conditioned_flags_are_rare_on_the_frame_workloads():
    for f in (synth.rgbd_120x160(), synth.lidar_64x1024()):
        r = oracle.extract_planes(f.points, oracle.OracleParams(**f.params), f.dominant_normals)
        assert r["ill_conditioned"].sum() <= 1e-4 * r["mask"].size


# ----------------------------------------------------------------------------- segment triangle lists


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_segment_lists_match_bucketing_by_hand(seed):
    """Section 7.2 takes each segment T^g_i as a triangle set: bucketing the labels GID by GID
    into a dict must give the same lists, segment order by label, triangles by T index."""
    rng = np.random.default_rng(seed)
    H, W = 9, 13
    pts = rng.normal(size=(H, W, 3)).astype(np.float32)
    pts[rng.random((H, W)) < 0.15] = np.nan
    T, Tmap = oracle.extract_triangles(oracle.widen(pts))
    n = 2 * (H - 1) * (W - 1)
    labels = np.full(n, -1, np.int32)
    valid = np.nonzero(Tmap >= 0)[0]
    roots = rng.choice(valid, size=5, replace=False)
    for g in valid:
        if rng.random() < 0.7:
            r = roots[rng.integers(0, 5)]
            labels[g] = min(r, g) if g < r else r   # any label; lists are defined for any values
    buckets = {}
    for g in range(n):
        if labels[g] >= 0:
            buckets.setdefault(int(labels[g]), []).append(int(Tmap[g]))
    seg_labels, offsets, tris = oracle.segment_lists(labels, Tmap)
    assert list(seg_labels) == sorted(buckets)
    assert offsets[0] == 0 and offsets[-1] == len(tris) == sum(len(v) for v in buckets.values())
    for k, lab in enumerate(seg_labels):
        assert list(tris[offsets[k]:offsets[k + 1]]) == buckets[int(lab)]
        assert np.all(np.diff(tris[offsets[k]:offsets[k + 1]]) > 0)


def test_segment_border_of_full_grid_is_its_perimeter():
    """One segment over a fully valid grid: its boundary half-edges are exactly the grid's
    perimeter edges, 2 (H-1) + 2 (W-1) of them, one per border half-edge of Algorithm 2."""
    H, W = 6, 9
    pts = np.zeros((H, W, 3), np.float32)
    pts[..., 0], pts[..., 1] = np.meshgrid(np.arange(W), np.arange(H))
    out = oracle.mesh_outputs(pts, np.zeros(2 * (H - 1) * (W - 1), np.int32))
    assert len(out["T"]) == 2 * (H - 1) * (W - 1)
    bits = np.unpackbits(out["border"][:, None], axis=1, bitorder="little")[:, :3]
    assert bits.sum() == 2 * (H - 1) + 2 * (W - 1)
    assert np.array_equal(bits.astype(bool), out["HE"].reshape(-1, 3) < 0)
    assert list(out["seg_labels"]) == [0] and list(out["seg_offsets"]) == [0, len(out["T"])]


def test_segment_border_between_two_segments():
    """Two segments split at a quad column: every half-edge of the dividing line is a boundary
    half-edge on both sides (2 per quad row), on top of the perimeter; unlabelled triangles have no
    boundary bits."""
    H, W = 5, 8
    pts = np.zeros((H, W, 3), np.float32)
    pts[..., 0], pts[..., 1] = np.meshgrid(np.arange(W), np.arange(H))
    Hq, Wq = H - 1, W - 1
    gid = np.arange(2 * Hq * Wq)
    v = (gid // 2) % Wq
    labels = np.where(v < 3, 0, 6).astype(np.int32)
    out = oracle.mesh_outputs(pts, labels)
    bits = np.unpackbits(out["border"][:, None], axis=1, bitorder="little")[:, :3]
    assert bits.sum() == 2 * Hq + 2 * Wq + 2 * Hq
    labels[v == Wq - 1] = -1                           # the last quad column belongs to no segment
    out = oracle.mesh_outputs(pts, labels)
    bits = np.unpackbits(out["border"][:, None], axis=1, bitorder="little")[:, :3]
    unl = np.nonzero(labels[np.nonzero(out["Tmap"] >= 0)[0]] < 0)[0]
    assert bits[unl].sum() == 0
    # the labelled region's perimeter (its right side now faces the unlabelled column) plus the
    # dividing line counted on both sides
    assert bits.sum() == (2 * Hq + 2 * (Wq - 1)) + 2 * Hq


@pytest.mark.parametrize("seed", range(3))
def test_segment_border_with_holes_matches_the_implicit_twins(seed):
    """With NaN holes T indices and GIDs part ways. A triangle's half-edge is a boundary one iff the
    triangle is labelled and the quad-grid neighbour across that edge (found from the vertex lists,
    not from HE) is missing, unlabelled or labelled otherwise."""
    rng = np.random.default_rng(70 + seed)
    H, W = 7, 9
    pts = affine_grid(H, W)
    pts[rng.random((H, W)) < 0.15] = np.nan
    n = 2 * (H - 1) * (W - 1)
    labels = rng.choice(np.array([-1, 0, 5, 9], np.int32), size=n)
    out = oracle.mesh_outputs(pts, labels)
    T = out["T"]
    gid_of = np.nonzero(out["Tmap"] >= 0)[0]
    owner = {}                                            # directed edge -> GID of its triangle
    for t, g in enumerate(gid_of):
        for e in range(3):
            owner[(int(T[t, e]), int(T[t, (e + 1) % 3]))] = int(g)
    bits = np.unpackbits(out["border"][:, None], axis=1, bitorder="little")[:, :3]
    for t, g in enumerate(gid_of):
        for e in range(3):
            a, b = int(T[t, e]), int(T[t, (e + 1) % 3])
            other = owner.get((b, a))
            want = labels[g] >= 0 and (other is None or labels[other] != labels[g])
            assert bits[t, e] == want, (t, e)


def test_pipeline_measures_edges_after_smoothing():
    """The whole path applies the l_max test to the smoothed points (Algorithm 4 after the
    Laplacian): a spike that smoothing pulls back keeps triangles the raw spike would reject."""
    P = affine_grid(6, 7)
    P[3, 3, 2] += 0.2
    p = oracle.OracleParams(lap_iters=5, max_edge=0.15, min_dot=0.5)
    r = oracle.extract_planes(P, p, np.array([[0.0, 0.0, -1.0]], np.float32), sensitivity=False)
    raw = oracle.widen(P)
    m_raw, _ = oracle.mask(raw, raw, 0.15)
    m_smooth, _ = oracle.mask(raw, r["smoothed"], 0.15)
    assert (m_raw == 0).sum() == 6 and m_smooth.all()   # the six triangles around the spike
    assert np.array_equal(r["mask"], m_smooth)


# ----------------------------------------------------------------------------- Algorithm 5, seeded


def _strip(nq):
    """One quad row: chain position p of each GID (second(v) at 2v, first(v) at 2v+1, the order the
    twins link them along the row) and centroids rising 0.1 m per chain position."""
    gid = np.arange(2 * nq)
    p = np.where(gid % 2 == 1, gid - 1, gid + 1)
    C = np.zeros((2 * nq, 3))
    C[:, 2] = 0.1 * p
    return C


def test_seeded_growing_hand_case():
    """Seeds in GID order with ptp_max = 0.25 m. Seed 0 (z 0.1) takes GIDs 1 (z 0.0), 3 (0.2) and
    2 (0.3) and stops at 5 (0.4); seed 4 (z 0.5) takes 5, 7, 6 and stops at 9; ... so the
    segments are the GIDs 4s .. 4s+3, labelled 4s. The pairwise test with the same limit joins
    every step of 0.1 m into one component instead: the seed-relative plane is what splits."""
    nq = 10
    H, W = 2, nq + 1
    C = _strip(nq)
    G = np.zeros(2 * nq, np.uint8)
    nd = np.array([[0.0, 0.0, 1.0]])
    labels, margin = oracle.label_seeded(G, H, W, C, nd, 0.25)
    assert list(labels) == [4 * (g // 4) for g in range(2 * nq)]
    assert abs(margin - 0.05) < 1e-12
    pair = oracle.label(G, H, W, C, nd, max_offset=0.25)
    assert np.all(pair == 0)
    dropped, _ = oracle.label_seeded(G, H, W, C, nd, 0.25, tri_min=4)
    assert np.all(dropped == -1)                          # |T^g_i| = 4 is not > 4
    kept, _ = oracle.label_seeded(G, H, W, C, nd, 0.25, tri_min=3)
    assert np.array_equal(kept, labels)


def test_seeded_growing_dropped_segment_stays_consumed():
    """A segment dropped by tri_min keeps its triangles: a later seed does not take them. One quad
    row, chain positions 0..7 at heights 0, 0, 0.25, 0.45, ... with ptp_max 0.3: seed 0 (position
    1) takes positions 0 and 2 (GIDs 1 and 3) and stops at 0.45; with tri_min 3 that segment of 3
    is dropped. Seed 2 (position 3, 0.45) then takes positions 3..7 but not GID 3 (0.25, within
    0.3 of it), which stays consumed. With tri_min 2 the first segment is kept."""
    nq = 4
    H, W = 2, nq + 1
    gid = np.arange(2 * nq)
    pos = np.where(gid % 2 == 1, gid - 1, gid + 1)
    z = np.array([0.0, 0.0, 0.25, 0.45, 0.45, 0.45, 0.45, 0.45])
    C = np.zeros((2 * nq, 3))
    C[:, 2] = z[pos]
    G = np.zeros(2 * nq, np.uint8)
    nd = np.array([[0.0, 0.0, 1.0]])
    dropped, _ = oracle.label_seeded(G, H, W, C, nd, 0.3, tri_min=3)
    assert list(dropped) == [-1, -1, 2, -1, 2, 2, 2, 2]
    kept, _ = oracle.label_seeded(G, H, W, C, nd, 0.3, tri_min=2)
    assert list(kept) == [0, 0, 2, 0, 2, 2, 2, 2]


def test_seeded_growing_without_limit_is_the_components():
    f = synth.rgbd_120x160()
    op = oracle.OracleParams(**f.params)
    ref = oracle.extract_planes(f.points, op, f.dominant_normals, sensitivity=False)
    seeded, _ = oracle.label_seeded(ref["groups"], f.H, f.W, ref["centroids"], ref["nd_unit"], 1e9)
    assert np.array_equal(seeded, ref["labels"])
    tight, _ = oracle.label_seeded(ref["groups"], f.H, f.W, ref["centroids"], ref["nd_unit"], 0.01)
    # a tighter slab only splits segments: every seeded segment lies inside one component
    lab = ref["labels"]
    for s in np.unique(tight[tight >= 0]):
        assert len(np.unique(lab[tight == s])) == 1
    assert len(np.unique(tight[tight >= 0])) > len(np.unique(lab[lab >= 0]))

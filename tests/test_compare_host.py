"""The acceptance check itself (`oracle/compare.py`), on the CPU: the oracle's own result, cast to
the device's FP32 types, passes with zero errors, and each planted deviation fails on the side of
its bound the parity bar puts it -- so a GPU parity test cannot pass by a lax checker."""
import numpy as np
import pytest

import oracle
from oracle import compare
import synth


@pytest.fixture(scope="module")
def case():
    f = synth.depth_camera_scene(24, 32, seed=9, n_boxes=2)
    p = oracle.OracleParams(**f.params)
    ref = oracle.extract_planes(f.points, p, f.dominant_normals)
    dev = dict(mask=ref["mask"].copy(), normals=ref["normals"].astype(np.float32), labels=ref["labels"].copy(),
               groups=ref["groups"].copy(), points=ref["smoothed"].astype(np.float32))
    return f, p, ref, dev


def _copy(dev):
    return {k: v.copy() for k, v in dev.items()}


def _run(case, dev, ref=None):
    f, p, r, _ = case
    H, W = f.points.shape[:2]
    return compare.compare(dev, r if ref is None else ref, p, H, W)


def _largest_segment(ref):
    seg, cnt = np.unique(ref["labels"][ref["labels"] >= 0], return_counts=True)
    return seg[cnt.argmax()]


def _rotate(n, t):
    """n turned by t radians about an axis perpendicular to it."""
    a = np.cross(n, [1.0, 0.0, 0.0])
    if np.linalg.norm(a) < 0.5:
        a = np.cross(n, [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    return n * np.cos(t) + np.cross(a, n) * np.sin(t)


def test_angle_by_hand():
    t = np.array([1e-7, 1e-4, 0.5, np.pi / 2, 3.0])
    a = np.tile([1.0, 0.0, 0.0], (len(t), 1))
    b = np.stack([np.cos(t), np.sin(t), np.zeros_like(t)], 1)
    np.testing.assert_allclose(compare.angle_rad(a, b), t, rtol=1e-12)   # exact at small angles too
    assert compare.angle_rad(a[:1], -a[:1])[0] == pytest.approx(np.pi)


def test_the_oracle_itself_passes(case):
    rep = _run(case, _copy(case[3]))
    assert rep["mask_mismatch"] == 0 and rep["label_mismatch"] == 0 and rep["group_mismatch"] == 0
    assert rep["normals_max_err_rad"] < 1e-6 and rep["points_max_err_m"] < 1e-6
    assert rep["segments"] > 1


def test_normal_bound(case):
    ref = case[2]
    well = ~np.isnan(ref["normals"][:, 0]) & ~ref["ill_conditioned"]
    i = int(np.nonzero(well)[0][len(np.nonzero(well)[0]) // 2])
    for t, ok in ((5e-5, True), (2e-4, False)):
        dev = _copy(case[3])
        dev["normals"][i] = _rotate(ref["normals"][i], t).astype(np.float32)
        if ok:
            assert _run(case, dev)["normals_max_err_rad"] == pytest.approx(t, rel=1e-2)
        else:
            with pytest.raises(AssertionError, match="normals off"):
                _run(case, dev)
    dev = _copy(case[3])
    dev["normals"][i] = np.nan
    with pytest.raises(AssertionError, match="NaN pattern"):
        _run(case, dev)


def test_point_bound(case):
    ref = case[2]
    ok = np.argwhere(~np.isnan(ref["smoothed"][..., 0]))
    u, v = ok[len(ok) // 2]
    for d, good in ((1e-5, True), (3e-5, False)):
        dev = _copy(case[3])
        dev["points"] = ref["smoothed"].copy()
        dev["points"][u, v, 1] += d
        if good:
            assert _run(case, dev)["points_max_err_m"] == pytest.approx(d, rel=1e-6)
        else:
            with pytest.raises(AssertionError, match="smoothed points"):
                _run(case, dev)


def test_mask_is_bit_exact_except_near_the_edge_threshold(case):
    ref = case[2]
    i = int(np.nonzero(ref["mask"] == 1)[0][5])
    dev = _copy(case[3])
    dev["mask"][i] = 0
    with pytest.raises(AssertionError, match="mask differs"):
        _run(case, dev)
    # the same flip on a triangle the oracle flags as near l_max is accepted
    r2 = dict(ref)
    r2["near_edge"] = ref["near_edge"].copy()
    r2["near_edge"][i] = True
    assert _run(case, dev, r2)["mask_mismatch"] == 1


def test_labels_are_bit_exact(case):
    ref = case[2]
    members = np.nonzero(ref["labels"] == _largest_segment(ref))[0]
    assert members.size > 1
    dev = _copy(case[3])
    dev["labels"][members[-1]] = -1                     # one triangle dropped from its segment
    with pytest.raises(AssertionError, match="labels differ"):
        _run(case, dev)
    dev = _copy(case[3])
    dev["labels"][members] = members[-1]                # same partition, not named by its smallest GID
    with pytest.raises(AssertionError, match="labels differ"):
        _run(case, dev)


def test_group_change_needs_a_flag_and_then_the_labels_follow_it(case):
    ref = case[2]
    i = int(np.nonzero(ref["labels"] == _largest_segment(ref))[0][0])
    dev = _copy(case[3])
    dev["groups"][i] = 255
    with pytest.raises(AssertionError, match="groups differ"):
        _run(case, dev)
    # flagged as a near tie: accepted, and the labels must be those of the substituted groups
    r2 = dict(ref)
    r2["near_tie"] = ref["near_tie"].copy()
    r2["near_tie"][i] = True
    G = ref["groups"].copy()
    G[i] = 255
    f = case[0]
    p = case[1]
    H, W = f.points.shape[:2]
    dev["labels"] = oracle.label(G, H, W, ref["centroids"], ref["nd_unit"], p.max_offset, p.min_triangles)
    rep = _run(case, dev, r2)
    assert rep["group_mismatch"] == 1 and rep["label_mismatch"] == 0
    dev["labels"] = ref["labels"].copy()                # the unsubstituted labels no longer match
    with pytest.raises(AssertionError, match="labels differ"):
        _run(case, dev, r2)


def test_near_threshold_flags_by_construction():
    """The flags that let a decision differ are set exactly where the quantity lies within NEAR of
    its threshold, never more widely. A noise-free affine plane does not move under the filters;
    every triangle's normal is (0, 0, -1) and its longest edge the quad diagonal."""
    H, W, h = 6, 7, 0.0625
    u, v = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    P = np.stack([0.25 + v * h, -0.5 + u * h, np.full_like(u, 2.0)], -1).astype(np.float32)
    diag = np.hypot(h, h)
    n_tri = 2 * (H - 1) * (W - 1)
    assert oracle.NEAR == 1e-5

    def flags(max_edge, dots):
        nd = np.array([[np.sqrt(1 - c * c), 0.0, -c] if k == 0 else [-np.sqrt(1 - c * c), 0.0, -c]
                       for k, c in enumerate(dots)])
        r = oracle.extract_planes(P, oracle.OracleParams(max_edge=max_edge, min_dot=0.95), nd, sensitivity=False)
        np.testing.assert_allclose(r["edge"], diag, rtol=0, atol=1e-15)
        np.testing.assert_allclose(r["normals"], np.tile([0.0, 0.0, -1.0], (n_tri, 1)), atol=1e-15)
        return r["near_edge"], r["near_dot"], r["near_tie"]

    e, d, t = flags(diag + 5e-6, [0.95 + 5e-6])
    assert e.all() and d.all() and not t.any()          # one dominant normal: no runner-up
    e, d, t = flags(diag + 5e-5, [0.95 + 5e-5])
    assert not e.any() and not d.any() and not t.any()
    e, d, t = flags(diag + 5e-5, [0.97, 0.97])          # two dominant normals at equal angles
    assert not e.any() and not d.any() and t.all()
    e, d, t = flags(diag + 5e-5, [0.97, 0.97 - 5e-5])
    assert not t.any()


def _ill_ref(ref, i, sens):
    r2 = dict(ref)
    r2["ill_conditioned"] = ref["ill_conditioned"].copy()
    r2["sensitivity"] = ref["sensitivity"].copy()
    r2["ill_conditioned"][i] = True
    r2["sensitivity"][i] = sens
    return r2


def _clear_triangle(case):
    """A grouped triangle of the largest segment whose decisions are far from every threshold."""
    f, p, ref, _ = case
    members = np.nonzero(ref["labels"] == _largest_segment(ref))[0]
    second = np.where(np.isfinite(ref["second"]), ref["second"], -2.0)
    far = (ref["best"][members] - p.min_dot > 1e-2) & (ref["best"][members] - second[members] > 2e-2)
    return int(members[far][0])


def test_ill_conditioned_normals_are_held_to_their_own_bound(case):
    """An ill-conditioned normal (sensitivity s > 2.5e-5 rad) may be off by ILL_FACTOR s, never
    less than 1e-4 and never more than ILL_CAP_RAD: an error beyond that fails."""
    ref = case[2]
    i = _clear_triangle(case)
    assert compare.ILL_FACTOR == 8.0 and compare.ILL_CAP_RAD == 1e-3
    r2 = _ill_ref(ref, i, 5e-5)                          # bound 4e-4 rad
    dev = _copy(case[3])
    dev["normals"][i] = _rotate(ref["normals"][i], 3e-4).astype(np.float32)
    rep = _run(case, dev, r2)
    assert rep["ill_conditioned"] >= 1 and rep["ill_conditioned_max_err_rad"] == pytest.approx(3e-4, rel=1e-2)
    assert rep["ill_conditioned_max_ratio"] == pytest.approx(6.0, rel=1e-2)
    dev["normals"][i] = _rotate(ref["normals"][i], 5e-4).astype(np.float32)
    with pytest.raises(AssertionError, match="ill-conditioned normals off"):
        _run(case, dev, r2)
    # however large the sensitivity, the bound stops at ILL_CAP_RAD
    r3 = _ill_ref(ref, i, 1e-2)
    dev["normals"][i] = _rotate(ref["normals"][i], 1e-2).astype(np.float32)
    with pytest.raises(AssertionError, match="ill-conditioned normals off"):
        _run(case, dev, r3)
    # and never below the ordinary 1e-4 rad
    r4 = _ill_ref(ref, i, 3e-6)
    dev["normals"][i] = _rotate(ref["normals"][i], 9e-5).astype(np.float32)
    _run(case, dev, r4)


def test_ill_conditioned_group_changes_only_near_a_threshold(case):
    """An ill-conditioned triangle's group may differ only where its bound reaches ang_min or the
    runner-up's dot; elsewhere a group flip fails, and an accepted flip needs the rerun labels."""
    f, p, ref, _ = case
    i = _clear_triangle(case)
    H, W = f.points.shape[:2]
    r2 = _ill_ref(ref, i, 5e-5)                          # bound 4e-4: best is 1e-2 from ang_min
    dev = _copy(case[3])
    dev["groups"][i] = 255
    with pytest.raises(AssertionError, match="groups differ"):
        _run(case, dev, r2)
    r3 = dict(r2)
    r3["best"] = ref["best"].copy()
    r3["best"][i] = p.min_dot + 3e-4                     # within the bound of ang_min
    G = ref["groups"].copy()
    G[i] = 255
    dev["labels"] = oracle.label(G, H, W, ref["centroids"], ref["nd_unit"], p.max_offset, p.min_triangles)
    rep = _run(case, dev, r3)
    assert rep["ill_conditioned_group_flagged"] == 1 and rep["group_mismatch"] == 1
    dev["labels"] = ref["labels"].copy()
    with pytest.raises(AssertionError, match="labels differ"):
        _run(case, dev, r3)
    r4 = dict(r2)
    r4["second"] = ref["second"].copy()
    r4["second"][i] = ref["best"][i] - 7e-4              # within twice the bound of the best dot
    dev["labels"] = oracle.label(G, H, W, ref["centroids"], ref["nd_unit"], p.max_offset, p.min_triangles)
    assert _run(case, dev, r4)["ill_conditioned_group_flagged"] == 1

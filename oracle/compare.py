"""Acceptance check of a device result against the FP64 oracle (test infrastructure only).

Bounds: smoothed points within 2e-5 m, normals within 1e-4 rad (angle from atan2(|a x b|, a . b)
in FP64), masks bit-exact, label partitions bit-exact (both sides label a segment by its
smallest GID, so equal partitions mean equal arrays).

FP32 and FP64 may take a different side of a threshold when the quantity sits within
oracle.NEAR of it: the longest edge against l_max, the best dot against ang_min, or the two
best dots against each other. Such triangles are flagged by the oracle; a mask or group
mismatch is accepted only on a flagged triangle, and the labels are then checked against the
oracle's region growing rerun with the device's groups substituted on the flagged triangles
only. The number of flagged triangles is reported.

A normal that the problem itself does not determine to FP32 precision -- the oracle's
sensitivity runs (every Laplacian update and bilateral sum perturbed by 2^-21 relative, two
seeds) move it by s > 2.5e-5 rad, a quarter of the bound -- is ill-conditioned. It is held to
its own bound instead of 1e-4 rad: ILL_FACTOR * s (the perturbation is about eight FP32 rounding
units per update, so an FP32 evaluation of the same steps moves the normal by a few s at most),
never below 1e-4 rad and never above ILL_CAP_RAD. Its group may differ only where that bound can
move the decision: its best dot within the bound of ang_min, or its two best dots within twice
the bound of each other (for unit vectors a dot moves by at most the angle); such triangles are
flagged like the near-threshold ones, every other group is bit-exact. The count of
ill-conditioned triangles, their largest error and its largest ratio to s are reported.
"""
from __future__ import annotations

import numpy as np

from . import FLAG_SEED_PTP as _FLAG_SEED_PTP
from . import label as _label
from . import label_seeded as _label_seeded

POINT_TOL_M = 2e-5
NORMAL_TOL_RAD = 1e-4
# bound of an ill-conditioned normal: ILL_FACTOR times its measured sensitivity, clamped to
# [NORMAL_TOL_RAD, ILL_CAP_RAD]
ILL_FACTOR = 8.0
ILL_CAP_RAD = 1e-3


def angle_rad(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cr, np.einsum("ij,ij->i", a, b))


def compare(dev: dict, ref: dict, params, H: int, W: int, point_tol=POINT_TOL_M, normal_tol=NORMAL_TOL_RAD) -> dict:
    """dev: numpy arrays mask [T] u8, normals [T,3] f32, labels [T] i32, optional groups [T] u8 and
    points [H,W,3] f32. ref: oracle.extract_planes(...). Returns a report; raises AssertionError on a
    violation of the bounds above."""
    rep: dict = {}
    n_tri = ref["mask"].shape[0]
    ill = ref.get("ill_conditioned", np.zeros(n_tri, bool))
    sens = np.asarray(ref.get("sensitivity", np.zeros(n_tri)), np.float64)
    ill_bound = np.clip(ILL_FACTOR * sens, normal_tol, ILL_CAP_RAD)
    # an ill-conditioned triangle's group may differ only where its bound can move the decision
    best, second = ref["best"], ref["second"]
    has_best = np.isfinite(best)
    has_second = has_best & np.isfinite(second)
    b0 = np.where(has_best, best, 0.0)
    ill_near = ill & has_best & ((np.abs(b0 - params.min_dot) < ill_bound) |
                                 (has_second & (b0 - np.where(has_second, second, 0.0) < 2.0 * ill_bound)))
    flagged = ref["near_edge"] | ref["near_dot"] | ref["near_tie"] | ill_near
    rep["flagged"] = int(flagged.sum())
    rep["ill_conditioned"] = int(ill.sum())
    rep["ill_conditioned_group_flagged"] = int(ill_near.sum())

    if dev.get("points") is not None:
        P = np.asarray(dev["points"], np.float64).reshape(H, W, 3)
        S = ref["smoothed"]
        nan_d, nan_r = np.isnan(P).any(-1), np.isnan(S).any(-1)
        assert np.array_equal(nan_d, nan_r), f"smoothed NaN pattern differs at {np.argwhere(nan_d != nan_r)[:5]}"
        err = np.abs(P - S)[~nan_r].max() if (~nan_r).any() else 0.0
        rep["points_max_err_m"] = float(err)
        assert err <= point_tol, f"smoothed points off by {err:.3g} m > {point_tol}"

    N = np.asarray(dev["normals"], np.float64).reshape(-1, 3)
    Nr = ref["normals"]
    nan_d, nan_r = np.isnan(N).any(-1), np.isnan(Nr).any(-1)
    assert np.array_equal(nan_d, nan_r), f"normal NaN pattern differs at {np.nonzero(nan_d != nan_r)[0][:5]}"
    ang_all = np.zeros(N.shape[0])
    if (~nan_r).any():
        ang_all[~nan_r] = angle_rad(N[~nan_r], Nr[~nan_r])
    well = ~nan_r & ~ill
    ang = ang_all[well]
    rep["normals_max_err_rad"] = float(ang.max()) if ang.size else 0.0
    rep["normals_over_tol"] = int((ang > normal_tol).sum())
    ill_n = ill & ~nan_r
    rep["ill_conditioned_max_err_rad"] = float(ang_all[ill_n].max()) if ill_n.any() else 0.0
    rep["ill_conditioned_max_ratio"] = (float((ang_all[ill_n] / np.maximum(sens[ill_n], 1e-300)).max())
                                        if ill_n.any() else 0.0)
    assert rep["normals_max_err_rad"] <= normal_tol, (
        f"normals off by {rep['normals_max_err_rad']:.3g} rad > {normal_tol} on {rep['normals_over_tol']} triangles")
    over = ill_n & (ang_all > ill_bound)
    assert not over.any(), (
        f"ill-conditioned normals off by more than their bound on {over.sum()} triangles, first "
        f"{np.nonzero(over)[0][:5]}: {ang_all[over][:5]} rad against {ill_bound[over][:5]}")

    m = np.asarray(dev["mask"]).reshape(-1)
    mm = m != ref["mask"]
    rep["mask_mismatch"] = int(mm.sum())
    assert not (mm & ~ref["near_edge"]).any(), f"mask differs on unflagged triangles {np.nonzero(mm & ~ref['near_edge'])[0][:5]}"

    lab = np.asarray(dev["labels"]).reshape(-1).astype(np.int64)
    G_ref = ref["groups"]
    if dev.get("groups") is not None:
        G = np.asarray(dev["groups"]).reshape(-1)
        gm = G != G_ref
        rep["group_mismatch"] = int(gm.sum())
        assert not (gm & ~flagged).any(), f"groups differ on unflagged triangles {np.nonzero(gm & ~flagged)[0][:5]}"
        G_sub = np.where(flagged, G, G_ref).astype(np.uint8)
    else:
        G_sub = G_ref
    if rep["flagged"] and dev.get("groups") is not None:
        if getattr(params, "flags", 0) & _FLAG_SEED_PTP:
            want, _ = _label_seeded(G_sub, H, W, ref["centroids"], ref["nd_unit"], params.max_offset,
                                    params.min_triangles)
        else:
            want = _label(G_sub, H, W, ref["centroids"], ref["nd_unit"], params.max_offset, params.min_triangles)
    else:
        want = ref["labels"]
    lm = lab != want
    rep["label_mismatch"] = int(lm.sum())
    assert not lm.any(), f"labels differ on {lm.sum()} triangles, first {np.nonzero(lm)[0][:5]}"
    rep["segments"] = int(len(np.unique(want[want >= 0])))
    return rep

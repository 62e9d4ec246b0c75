"""FP64 CPU oracle for the organized-point-cloud plane-extraction path.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this package. The CUDA
library never calls it and shares no code with it.

The arithmetic lives in ``pl3d_oracle.c`` (plain C, double precision, loops in
the paper's order); this module compiles it with gcc, loads it through ctypes
and chains the steps the way the paper orders them:

    Laplacian (Eq. 1-2) -> centroids/normals over T_FC (Section 5.2)
    -> bilateral normal filter (Eq. 3-6) -> mask (Algorithm 1 + Algorithm 4's
    edge predicate) -> group assignment (Algorithm 4) -> region growing
    (Algorithm 5 over the twins of Algorithm 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pl3d_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lib = None

_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available) into liborc.so."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", _SRC, "-o", _LIB_PATH + ".tmp"]
    try:
        subprocess.run(base[:6] + ["-fopenmp"] + base[6:] + ["-lm"], check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True, text=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_get_threads.restype = ctypes.c_int
    lib.orc_has_openmp.restype = ctypes.c_int
    lib.orc_widen.argtypes = [_f32p, ctypes.c_int64, _f64p]
    lib.orc_laplacian.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _f64p]
    lib.orc_laplacian_jitter.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_uint64, _f64p]
    lib.orc_bilateral_jitter.argtypes = [_f64p, _f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, _f64p]
    lib.orc_triangle_geometry.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, _f64p, _f64p]
    lib.orc_mask.argtypes = [_f64p, _f64p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _u8p, _f64p]
    lib.orc_bilateral.argtypes = [_f64p, _f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_int, _f64p]
    lib.orc_normalize_dominant.argtypes = [_f32p, ctypes.c_int, _f64p]
    lib.orc_classify.argtypes = [_f64p, _u8p, ctypes.c_int64, _f64p, ctypes.c_int, ctypes.c_double, _u8p, _f64p, _f64p]
    lib.orc_triangle_twins.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, _i64p]
    lib.orc_label.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _f64p, _f64p, ctypes.c_int, ctypes.c_double,
                              ctypes.c_int, _i32p]
    lib.orc_label_seeded.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _f64p, _f64p, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, _i32p, _f64p]
    lib.orc_extract_triangles.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, _i32p, _i32p]
    lib.orc_extract_triangles.restype = ctypes.c_int64
    lib.orc_extract_halfedges.argtypes = [_i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _i32p]
    for name in ("orc_laplacian", "orc_laplacian_jitter", "orc_bilateral_jitter", "orc_triangle_geometry", "orc_mask", "orc_bilateral", "orc_normalize_dominant",
                 "orc_classify", "orc_label", "orc_label_seeded", "orc_extract_halfedges", "orc_triangle_twins"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _check(rc: int, what: str):
    if rc < 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def has_openmp() -> bool:
    return bool(_load().orc_has_openmp())


# --------------------------------------------------------------------------- steps


def widen(points: np.ndarray) -> np.ndarray:
    """FP32 [H, W, 3] -> FP64 [H, W, 3]; a point with any non-finite coordinate becomes NaN (Section 4.2)."""
    pts = np.ascontiguousarray(points, dtype=np.float32)
    out = np.empty(pts.shape, dtype=np.float64)
    _load().orc_widen(_p(pts, _f32p), pts.size // 3, _p(out, _f64p))
    return out


def laplacian(P: np.ndarray, kernel: int, lam: float, iters: int, eps: float = 0.0, seed: int = 0) -> np.ndarray:
    """Eq. 1-2 / Section 5.1: `iters` Jacobi iterations of the Laplacian filter on FP64 [H, W, 3].
    eps > 0 scales every update by (1 +- eps) (seeded signs): a sensitivity run, not the method."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    H, W = P.shape[:2]
    out = np.empty_like(P)
    _check(_load().orc_laplacian_jitter(_p(P, _f64p), H, W, kernel, lam, iters, float(eps), int(seed),
                                        _p(out, _f64p)), "laplacian")
    return out


def triangle_geometry(P: np.ndarray):
    """Section 5.2: centroids C and unit normals N over T_FC, both FP64 [2(H-1)(W-1), 3]."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    H, W = P.shape[:2]
    n = 2 * (H - 1) * (W - 1)
    C = np.empty((n, 3), np.float64)
    N = np.empty((n, 3), np.float64)
    _check(_load().orc_triangle_geometry(_p(P, _f64p), H, W, _p(C, _f64p), _p(N, _f64p)), "geometry")
    return C, N


def mask(P_raw: np.ndarray, P_smooth: np.ndarray, l_max: float):
    """Algorithm 1 validity and Algorithm 4's edge predicate -> (uint8 mask, FP64 longest edge)."""
    P_raw = np.ascontiguousarray(P_raw, dtype=np.float64)
    P_smooth = np.ascontiguousarray(P_smooth, dtype=np.float64)
    H, W = P_raw.shape[:2]
    n = 2 * (H - 1) * (W - 1)
    m = np.empty(n, np.uint8)
    e = np.empty(n, np.float64)
    _check(_load().orc_mask(_p(P_raw, _f64p), _p(P_smooth, _f64p), H, W, l_max, _p(m, _u8p), _p(e, _f64p)), "mask")
    return m, e


def bilateral(C: np.ndarray, N: np.ndarray, H: int, W: int, kernel: int, sigma_c: float, sigma_s: float,
              iters: int, eps: float = 0.0, seed: int = 0) -> np.ndarray:
    """Eq. 3-6 / Section 5.2: `iters` Jacobi iterations of the bilateral normal filter.
    eps > 0 scales every weighted sum by (1 +- eps) per coordinate (sensitivity run)."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    N = np.ascontiguousarray(N, dtype=np.float64)
    out = np.empty_like(N)
    _check(_load().orc_bilateral_jitter(_p(C, _f64p), _p(N, _f64p), H, W, kernel, sigma_c, sigma_s, iters,
                                        float(eps), int(seed), _p(out, _f64p)), "bilateral")
    return out


def normalize_dominant(nd: np.ndarray) -> np.ndarray:
    nd32 = np.ascontiguousarray(nd, dtype=np.float32).reshape(-1, 3)
    out = np.empty(nd32.shape, np.float64)
    _check(_load().orc_normalize_dominant(_p(nd32, _f32p), nd32.shape[0], _p(out, _f64p)), "normalize")
    return out


def classify(N: np.ndarray, m: np.ndarray, nd_unit: np.ndarray, ang_min: float):
    """Algorithm 4 -> (uint8 groups, best dot, second-best dot)."""
    N = np.ascontiguousarray(N, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.uint8)
    nd_unit = np.ascontiguousarray(nd_unit, dtype=np.float64)
    n = m.shape[0]
    G = np.empty(n, np.uint8)
    best = np.empty(n, np.float64)
    second = np.empty(n, np.float64)
    _check(_load().orc_classify(_p(N, _f64p), _p(m, _u8p), n, _p(nd_unit, _f64p), nd_unit.shape[0], ang_min,
                                _p(G, _u8p), _p(best, _f64p), _p(second, _f64p)), "classify")
    return G, best, second


def label(G: np.ndarray, H: int, W: int, C=None, nd_unit=None, max_offset: float = 0.0, tri_min: int = 0):
    """Algorithm 5 over Algorithm 2's twins -> int32 labels (min GID of the component, -1 = none)."""
    G = np.ascontiguousarray(G, dtype=np.uint8)
    out = np.empty(G.shape[0], np.int32)
    Cp = _p(np.ascontiguousarray(C, dtype=np.float64), _f64p) if C is not None else None
    nd = np.ascontiguousarray(nd_unit, dtype=np.float64) if nd_unit is not None else None
    K = nd.shape[0] if nd is not None else 0
    _check(_load().orc_label(_p(G, _u8p), H, W, Cp, _p(nd, _f64p) if nd is not None else None, K,
                             float(max_offset), int(tri_min), _p(out, _i32p)), "label")
    return out


def label_seeded(G: np.ndarray, H: int, W: int, C: np.ndarray, nd_unit: np.ndarray, ptp_max: float,
                 tri_min: int = 0):
    """Algorithm 5 with the seed-relative point-to-plane limit (seeds in GID order)
    -> (int32 labels, smallest |offset - ptp_max| over the tests made)."""
    G = np.ascontiguousarray(G, dtype=np.uint8)
    out = np.empty(G.shape[0], np.int32)
    C = np.ascontiguousarray(C, dtype=np.float64)
    nd = np.ascontiguousarray(nd_unit, dtype=np.float64)
    margin = np.zeros(1, np.float64)
    _check(_load().orc_label_seeded(_p(G, _u8p), H, W, _p(C, _f64p), _p(nd, _f64p), nd.shape[0], float(ptp_max),
                                    int(tri_min), _p(out, _i32p), _p(margin, _f64p)), "label_seeded")
    return out, float(margin[0])


def triangle_twins(gid: int, H: int, W: int):
    buf = np.empty(3, np.int64)
    n = _load().orc_triangle_twins(int(gid), H, W, _p(buf, _i64p))
    return [int(x) for x in buf[:n]]


def extract_triangles(P_raw: np.ndarray):
    """Algorithm 1 -> (T int32 [n, 3] point indices, T_map int32 [2(H-1)(W-1)])."""
    P_raw = np.ascontiguousarray(P_raw, dtype=np.float64)
    H, W = P_raw.shape[:2]
    n = 2 * (H - 1) * (W - 1)
    T = np.empty((max(n, 1), 3), np.int32)
    Tmap = np.empty(n, np.int32)
    ntri = _load().orc_extract_triangles(_p(P_raw, _f64p), H, W, _p(T, _i32p), _p(Tmap, _i32p))
    _check(int(ntri), "extract_triangles")
    return T[:ntri].copy(), Tmap


def extract_halfedges(Tmap: np.ndarray, H: int, W: int, ntri: int) -> np.ndarray:
    """Algorithm 2 -> HE int32 [3 ntri] (twin half-edge id or -1)."""
    Tmap = np.ascontiguousarray(Tmap, dtype=np.int32)
    HE = np.empty(max(3 * ntri, 1), np.int32)
    _check(_load().orc_extract_halfedges(_p(Tmap, _i32p), H, W, int(ntri), _p(HE, _i32p)), "extract_halfedges")
    return HE[:3 * ntri].copy()


def segment_lists(labels: np.ndarray, Tmap: np.ndarray):
    """Planar segments as triangle sets (Algorithm 5's output T^g_i, the input of polygon
    extraction, Section 7.2). Segments are ordered by label (their smallest GID); each holds the
    T indices (Algorithm 1) of its triangles in ascending order.
    -> (seg_labels int32 [S], offsets int32 [S + 1], tris int32 [offsets[S]])."""
    labels = np.asarray(labels, np.int64)
    Tmap = np.asarray(Tmap, np.int64)
    gids = np.nonzero(labels >= 0)[0]                    # ascending GID
    lab = labels[gids]
    order = np.argsort(lab, kind="stable")               # by label, ties kept in GID order
    seg_labels, counts = np.unique(lab, return_counts=True)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return seg_labels.astype(np.int32), offsets, Tmap[gids[order]].astype(np.int32)


def segment_border(T_labels: np.ndarray, HE: np.ndarray) -> np.ndarray:
    """Boundary half-edges of the segments (the set BE of Section 7.2): bit e of entry t is set when
    triangle t belongs to a segment and its half-edge 3t + e has no twin (HE = -1) or a twin whose
    triangle carries another label. -> uint8 [len(T_labels)]."""
    T_labels = np.asarray(T_labels, np.int64)
    HE = np.asarray(HE, np.int64).reshape(-1, 3)
    out = np.zeros(len(T_labels), np.uint8)
    for e in range(3):
        tw = HE[:, e]
        other = np.where(tw >= 0, T_labels[np.maximum(tw, 0) // 3], -2)
        border = (T_labels >= 0) & ((tw < 0) | (other != T_labels))
        out |= (border.astype(np.uint8) << e)
    return out


def mesh_outputs(points: np.ndarray, labels: np.ndarray) -> dict:
    """Explicit mesh (Algorithm 1: T, T_map; Algorithm 2: HE) of a frame and its segments' triangle
    lists and boundary half-edges, given the frame's labels."""
    H, W = points.shape[:2]
    T, Tmap = extract_triangles(widen(points))
    HE = extract_halfedges(Tmap, H, W, len(T))
    seg_labels, offsets, tris = segment_lists(labels, Tmap)
    gid_of = np.nonzero(np.asarray(Tmap) >= 0)[0]      # T index -> GID (T keeps GID order)
    T_labels = np.asarray(labels)[gid_of]
    return dict(T=T, Tmap=Tmap, HE=HE, seg_labels=seg_labels, seg_offsets=offsets, seg_tris=tris,
                border=segment_border(T_labels, HE))


# --------------------------------------------------------------------------- pipeline


@dataclass
class OracleParams:
    """The oracle's own copy of the method's parameters (paper notation in comments)."""
    lap_iters: int = 5
    lap_lambda: float = 1.0        # lambda, Eq. 1
    lap_kernel: int = 3
    bil_iters: int = 3
    bil_sigma_len: float = 0.1     # sigma_c, Eq. 4
    bil_sigma_ang: float = 0.15    # sigma_s, Eq. 5
    bil_kernel: int = 3
    max_edge: float = 0.1          # l_max, Algorithm 4 (<= 0 disables)
    min_dot: float = 0.95          # ang_min, Algorithm 4
    max_offset: float = 0.0        # pairwise plane-offset join test (<= 0 disables), or ptp_max
    min_triangles: int = 0         # tri_min, Algorithm 5 (0 disables)
    flags: int = 0                 # FLAG_SEED_PTP: max_offset is Algorithm 5's seed-relative ptp_max


# flags bit: region growing with the seed-relative point-to-plane limit (Algorithm 5) instead of
# the order-independent pairwise offset test
FLAG_SEED_PTP = 1


# Width of the band around a threshold inside which FP32 and FP64 may decide differently.
NEAR = 1e-5
# Relative size of the perturbation used to find outputs that FP32 arithmetic cannot pin down
# (a few units of FP32 rounding, 2^-21, applied to every update of every iteration), the seeds
# of the runs (the largest move over the runs counts), and the angle a normal may move under it
# before the triangle counts as ill-conditioned (a quarter of the 1e-4 rad acceptance bound).
JITTER = 2.0 ** -21
JITTER_SEEDS = (0x5EED, 0xB11A)
ILL_CONDITIONED_RAD = 2.5e-5


def _angle(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cr, np.einsum("ij,ij->i", a, b))


def extract_planes(points: np.ndarray, params, dominant_normals: np.ndarray, sensitivity: bool = True) -> dict:
    """The whole path in the paper's order. Returns every intermediate, FP64 where real-valued.

    Keys: smoothed [H,W,3], centroids [T,3], normals_raw [T,3], normals [T,3], mask [T] u8,
    edge [T], groups [T] u8, best [T], second [T], labels [T] i32, nd_unit [K,3],
    near_edge / near_dot / near_tie [T] bool (decisions within NEAR of a threshold),
    sensitivity [T] FP64 (sensitivity=True: the largest angle by which the normal moves when the
    Laplacian updates and bilateral sums are perturbed by JITTER relative, over the JITTER_SEEDS
    runs; 0 without a normal), ill_conditioned [T] bool (sensitivity > ILL_CONDITIONED_RAD: FP32
    arithmetic cannot be expected to reproduce that normal to the 1e-4 rad bound).
    """
    p = params
    H, W = points.shape[:2]
    raw = widen(points)
    smoothed = laplacian(raw, p.lap_kernel, p.lap_lambda, p.lap_iters)
    C, N0 = triangle_geometry(smoothed)
    N = bilateral(C, N0, H, W, p.bil_kernel, p.bil_sigma_len, p.bil_sigma_ang, p.bil_iters)
    m, edge = mask(raw, smoothed, p.max_edge)
    nd_unit = normalize_dominant(dominant_normals)
    G, best, second = classify(N, m, nd_unit, p.min_dot)
    ptp_margin = None
    if p.flags & FLAG_SEED_PTP:
        labels, ptp_margin = label_seeded(G, H, W, C, nd_unit, p.max_offset, p.min_triangles)
    else:
        labels = label(G, H, W, C, nd_unit, p.max_offset, p.min_triangles)
    finite_edge = np.isfinite(edge)
    near_edge = finite_edge & (np.abs(np.where(finite_edge, edge, 0.0) - p.max_edge) < NEAR) & (p.max_edge > 0)
    has_best = np.isfinite(best)
    near_dot = has_best & (np.abs(np.where(has_best, best, 0.0) - p.min_dot) < NEAR)
    has_second = has_best & np.isfinite(second)
    near_tie = has_second & ((np.where(has_second, best - second, 1.0)) < NEAR)
    ill = np.zeros(m.shape[0], bool)
    ang = np.zeros(m.shape[0])
    if sensitivity:
        for seed in JITTER_SEEDS:
            Sj = laplacian(raw, p.lap_kernel, p.lap_lambda, p.lap_iters, JITTER, seed)
            Cj, Nj0 = triangle_geometry(Sj)
            Nj = bilateral(Cj, Nj0, H, W, p.bil_kernel, p.bil_sigma_len, p.bil_sigma_ang, p.bil_iters, JITTER,
                           seed + 1)
            has = ~np.isnan(N[:, 0]) & ~np.isnan(Nj[:, 0])
            ang[has] = np.maximum(ang[has], _angle(N[has], Nj[has]))
        ill = ang > ILL_CONDITIONED_RAD
    return dict(smoothed=smoothed, centroids=C, normals_raw=N0, normals=N, mask=m, edge=edge, groups=G,
                best=best, second=second, labels=labels, nd_unit=nd_unit, near_edge=near_edge,
                near_dot=near_dot, near_tie=near_tie, ill_conditioned=ill, sensitivity=ang, ptp_margin=ptp_margin)

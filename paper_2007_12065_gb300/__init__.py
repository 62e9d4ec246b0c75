"""pl3d -- GB300 (sm_103a) plane extraction for organized point clouds, after Polylidar3D.

Thin ctypes binding over libpl3d.so (the C ABI in include/pl3d.h). Each function here has the
name of the C entry point it calls and does argument marshalling only: every step of the path
runs in the library's CUDA kernels. PyTorch is used for device memory and streams.

The library must have been built (``__graft_entry__.build()`` or
``python paper_2007_12065_gb300/build.py``); calls fail loudly when it is missing -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpl3d.so")

PL3D_OK = 0
PL3D_ERR_INVALID_ARG = -1
PL3D_ERR_OUT_OF_MEMORY = -2
PL3D_ERR_CUDA = -3
PL3D_ERR_TIMEOUT = -4
PL3D_ERR_UNSUPPORTED = -5
PL3D_MAX_GROUPS = 254
PL3D_NO_GROUP = 255
PL3D_TIMING_SLOTS = 13
PL3D_FLAG_SEED_PTP = 1


class pl3d_params(ctypes.Structure):
    """Mirror of the C struct pl3d_params (field meaning documented in include/pl3d.h)."""
    _fields_ = [
        ("lap_iters", ctypes.c_int32),
        ("lap_lambda", ctypes.c_float),
        ("lap_kernel", ctypes.c_int32),
        ("bil_iters", ctypes.c_int32),
        ("bil_sigma_len", ctypes.c_float),
        ("bil_sigma_ang", ctypes.c_float),
        ("bil_kernel", ctypes.c_int32),
        ("max_edge", ctypes.c_float),
        ("min_dot", ctypes.c_float),
        ("max_offset", ctypes.c_float),
        ("min_triangles", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class pl3d_frame(ctypes.Structure):
    """Mirror of the C struct pl3d_frame: one frame of a batch."""
    _fields_ = [
        ("points", ctypes.c_void_p),
        ("H", ctypes.c_int32),
        ("W", ctypes.c_int32),
        ("params", ctypes.POINTER(pl3d_params)),
        ("dominant_normals", ctypes.c_void_p),
        ("K", ctypes.c_int32),
        ("out_tri_mask", ctypes.c_void_p),
        ("out_normals", ctypes.c_void_p),
        ("out_labels", ctypes.c_void_p),
        ("out_points", ctypes.c_void_p),
        ("out_groups", ctypes.c_void_p),
    ]


class pl3d_tuning(ctypes.Structure):
    """Mirror of the C struct pl3d_tuning (launch shape; never changes a result)."""
    _fields_ = [
        ("lap_fuse", ctypes.c_int32),
        ("bil_fuse", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("lap_tile_h", ctypes.c_int32),
        ("bil_tile_h", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class pl3d_server_config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int32),
        ("max_inflight", ctypes.c_int32),
        ("max_batch_frames", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("hbm_bytes", ctypes.c_int64),
    ]


class pl3d_completion(ctypes.Structure):
    _fields_ = [
        ("ticket", ctypes.c_uint64),
        ("status", ctypes.c_int32),
        ("batch_frames", ctypes.c_int32),
        ("latency_ms", ctypes.c_double),
        ("queue_ms", ctypes.c_double),
    ]


class pl3d_server_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in ("submitted", "completed", "rejected", "batches", "triangles",
                                                   "max_batch_frames", "max_inflight", "slot_bytes")]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class pl3d_replay_source(ctypes.Structure):
    """Mirror of the C struct pl3d_replay_source (one sensor of a trace replay)."""
    _fields_ = [
        ("host_points", ctypes.POINTER(ctypes.c_void_p)),
        ("n_variants", ctypes.c_int32),
        ("H", ctypes.c_int32),
        ("W", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("params", ctypes.POINTER(pl3d_params)),
        ("dominant_normals", ctypes.c_void_p),
        ("ring", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("host_mask", ctypes.POINTER(ctypes.c_void_p)),
        ("host_normals", ctypes.POINTER(ctypes.c_void_p)),
        ("host_labels", ctypes.POINTER(ctypes.c_void_p)),
    ]


class pl3d_replay_report(ctypes.Structure):
    _fields_ = ([(name, ctypes.c_int64) for name in ("requests", "completed", "failed", "batches", "max_batch_frames",
                                                     "max_inflight")] +
                [(name, ctypes.c_double) for name in ("seconds", "p50_ms", "p90_ms", "p99_ms", "max_ms", "mean_ms",
                                                      "mtri_s", "achieved_fps", "mean_batch_frames",
                                                      "submit_lag_p99_ms")])

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class PL3DError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {pl3d_status_string(status)} ({status})")
        self.status = status


_lib = None
_vp = ctypes.c_void_p


def lib():
    """The loaded libpl3d.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the plane-extraction path has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(pl3d_params)
    L.pl3d_version.restype = ctypes.c_int
    L.pl3d_status_string.argtypes = [ctypes.c_int]
    L.pl3d_status_string.restype = ctypes.c_char_p
    L.pl3d_timing_slot_name.argtypes = [ctypes.c_int]
    L.pl3d_timing_slot_name.restype = ctypes.c_char_p
    L.pl3d_default_params.argtypes = [P]
    L.pl3d_validate.argtypes = [P, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]
    L.pl3d_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
    L.pl3d_destroy.argtypes = [_vp]
    L.pl3d_destroy.restype = None
    L.pl3d_extract_planes.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, P, _vp, ctypes.c_int, _vp, _vp, _vp, _vp]
    L.pl3d_extract_planes_ex.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, P, _vp, ctypes.c_int, _vp, _vp, _vp,
                                         _vp, _vp, _vp]
    L.pl3d_extract_planes_host.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, P, _vp, ctypes.c_int, _vp, _vp, _vp,
                                           _vp]
    L.pl3d_sync.argtypes = [_vp, _vp]
    L.pl3d_set_timing.argtypes = [_vp, ctypes.c_int]
    L.pl3d_read_timing.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int]
    L.pl3d_launch_count.argtypes = [_vp]
    L.pl3d_launch_count.restype = ctypes.c_int64
    L.pl3d_extract_planes_static.argtypes = [_vp, ctypes.c_int, ctypes.c_int, P, _vp, ctypes.c_int, _vp, _vp, _vp, _vp]
    L.pl3d_static_scratch_bytes.restype = ctypes.c_size_t
    L.pl3d_static_sync.argtypes = [_vp]
    L.pl3d_selftest_wait_timeout.argtypes = [_vp, ctypes.c_int, ctypes.c_int64, _vp]
    F = ctypes.POINTER(pl3d_frame)
    T = ctypes.POINTER(pl3d_tuning)
    L.pl3d_extract_planes_batched.argtypes = [_vp, F, ctypes.c_int, _vp]
    L.pl3d_set_tuning.argtypes = [_vp, T]
    L.pl3d_get_tuning.argtypes = [_vp, T]
    L.pl3d_autotune_batched.argtypes = [_vp, F, ctypes.c_int, _vp, ctypes.c_int, T, ctypes.POINTER(ctypes.c_double)]
    L.pl3d_batch_stats.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)]
    L.pl3d_extract_mesh.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                    _vp]
    L.pl3d_fastga_cells.argtypes = [ctypes.c_int, _vp, _vp]
    L.pl3d_fastga.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]
    L.pl3d_fastga_peaks.argtypes = [ctypes.c_int, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_int, _vp, _vp]
    L.pl3d_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(pl3d_server_config)]
    L.pl3d_server_submit.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, P, _vp, ctypes.c_int, _vp, _vp, _vp,
                                     ctypes.POINTER(ctypes.c_uint64)]
    L.pl3d_server_poll.argtypes = [_vp, ctypes.POINTER(pl3d_completion), ctypes.c_int, ctypes.c_int]
    L.pl3d_server_drain.argtypes = [_vp]
    L.pl3d_server_get_stats.argtypes = [_vp, ctypes.POINTER(pl3d_server_stats)]
    L.pl3d_server_destroy.argtypes = [_vp]
    L.pl3d_server_destroy.restype = None
    L.pl3d_server_replay.argtypes = [_vp, ctypes.POINTER(pl3d_replay_source), ctypes.c_int, _vp, _vp, ctypes.c_int64,
                                     ctypes.POINTER(pl3d_replay_report)]
    L.pl3d_pipeline_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(_vp)]
    L.pl3d_pipeline_submit.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, P, _vp, ctypes.c_int, _vp, _vp, _vp,
                                       ctypes.POINTER(ctypes.c_uint64)]
    L.pl3d_pipeline_wait.argtypes = [_vp, ctypes.c_uint64]
    L.pl3d_pipeline_destroy.argtypes = [_vp]
    L.pl3d_pipeline_context.argtypes = [_vp]
    L.pl3d_pipeline_context.restype = _vp
    _lib = L
    return L


# ----------------------------------------------------------------------------- marshalling helpers


def _ptr(x) -> Optional[int]:
    """Address of a torch tensor, a numpy array, an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _nd_host(dominant_normals, K: Optional[int] = None):
    """Dominant normals as a contiguous host float32 buffer (kept alive by the caller); with K,
    the buffer must hold at least K rows, since the library reads K * 3 floats from it."""
    import numpy as np
    if hasattr(dominant_normals, "detach"):
        dominant_normals = dominant_normals.detach().cpu().numpy()
    nd = np.ascontiguousarray(dominant_normals, dtype=np.float32).reshape(-1, 3)
    if K is not None and int(K) > nd.shape[0]:
        raise ValueError(f"K = {int(K)} but dominant_normals holds {nd.shape[0]} normals")
    return nd


def _check(status: int, what: str) -> int:
    if status != PL3D_OK:
        raise PL3DError(status, what)
    return status


def _check_tensor(t, name, dtype, numel, device_kind="cuda"):
    """A torch tensor on the right device, or (host buffers only) a numpy array, contiguous, of
    the right dtype and element count. Raw int addresses are passed through unchecked."""
    if t is None:
        return
    if hasattr(t, "is_cuda"):
        if (device_kind == "cuda") != t.is_cuda:
            raise ValueError(f"{name} must be a {device_kind} tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if str(t.dtype) != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if t.numel() != numel:
            raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    elif hasattr(t, "__array_interface__"):
        if device_kind == "cuda":
            raise ValueError(f"{name} must be a cuda tensor, got a host array")
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name} must be contiguous")
        if str(t.dtype) != dtype.split(".")[-1]:
            raise ValueError(f"{name} must be {dtype.split('.')[-1]}, got {t.dtype}")
        if t.size != numel:
            raise ValueError(f"{name} must have {numel} elements, got {t.size}")


# ----------------------------------------------------------------------------- the C ABI, by name


def pl3d_version() -> int:
    return int(lib().pl3d_version())


def pl3d_status_string(status: int) -> str:
    return lib().pl3d_status_string(int(status)).decode()


def pl3d_timing_slot_name(slot: int) -> str:
    return lib().pl3d_timing_slot_name(int(slot)).decode()


def pl3d_default_params() -> pl3d_params:
    p = pl3d_params()
    _check(lib().pl3d_default_params(ctypes.byref(p)), "pl3d_default_params")
    return p


def make_params(**kw) -> pl3d_params:
    """pl3d_params from keyword arguments (paper-named fields); unspecified fields take the defaults."""
    p = pl3d_default_params()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(f"unknown parameter {k!r}")
        setattr(p, k, v)
    return p


def pl3d_validate(params: pl3d_params, H: int, W: int, dominant_normals=None, K: Optional[int] = None) -> int:
    """Host-only argument check; returns the status code (0 = valid)."""
    nd = _nd_host(dominant_normals) if dominant_normals is not None else None
    if K is None:
        K = nd.shape[0] if nd is not None else 1
    if nd is not None and int(K) > nd.shape[0]:
        return PL3D_ERR_INVALID_ARG   # the library would read K normals from a shorter buffer
    return int(lib().pl3d_validate(ctypes.byref(params), int(H), int(W), _ptr(nd), int(K)))


def pl3d_create(device: int = 0) -> int:
    """Creates a context on `device`; returns its handle (an address)."""
    h = _vp()
    _check(lib().pl3d_create(ctypes.byref(h), int(device)), "pl3d_create")
    return int(h.value)


def pl3d_destroy(ctx: int) -> None:
    lib().pl3d_destroy(ctx)


def pl3d_extract_planes(ctx, points, H, W, params, dominant_normals, K, out_tri_mask, out_normals, out_labels,
                        stream=None) -> int:
    """Device buffers (torch CUDA tensors or raw addresses); see include/pl3d.h."""
    return pl3d_extract_planes_ex(ctx, points, H, W, params, dominant_normals, K, out_tri_mask, out_normals,
                                  out_labels, None, None, stream)


def pl3d_extract_planes_ex(ctx, points, H, W, params, dominant_normals, K, out_tri_mask, out_normals, out_labels,
                           out_points=None, out_groups=None, stream=None) -> int:
    n_tri = 2 * (H - 1) * (W - 1)
    _check_tensor(points, "points", "torch.float32", H * W * 3)
    _check_tensor(out_tri_mask, "out_tri_mask", "torch.uint8", n_tri)
    _check_tensor(out_normals, "out_normals", "torch.float32", n_tri * 3)
    _check_tensor(out_labels, "out_labels", "torch.int32", n_tri)
    _check_tensor(out_points, "out_points", "torch.float32", H * W * 3)
    _check_tensor(out_groups, "out_groups", "torch.uint8", n_tri)
    nd = _nd_host(dominant_normals, K)
    return _check(lib().pl3d_extract_planes_ex(ctx, _ptr(points), int(H), int(W), ctypes.byref(params), _ptr(nd),
                                               int(K), _ptr(out_tri_mask), _ptr(out_normals), _ptr(out_labels),
                                               _ptr(out_points), _ptr(out_groups), _stream(stream)),
                  "pl3d_extract_planes")


def pl3d_extract_planes_host(ctx, points, H, W, params, dominant_normals, K, out_tri_mask, out_normals, out_labels,
                             stream=None) -> int:
    """Host buffers (CPU tensors, pinned for async DMA, or numpy arrays); synchronises before returning."""
    n_tri = 2 * (H - 1) * (W - 1)
    _check_tensor(points, "points", "torch.float32", H * W * 3, "cpu")
    _check_tensor(out_tri_mask, "out_tri_mask", "torch.uint8", n_tri, "cpu")
    _check_tensor(out_normals, "out_normals", "torch.float32", n_tri * 3, "cpu")
    _check_tensor(out_labels, "out_labels", "torch.int32", n_tri, "cpu")
    nd = _nd_host(dominant_normals, K)
    return _check(lib().pl3d_extract_planes_host(ctx, _ptr(points), int(H), int(W), ctypes.byref(params), _ptr(nd),
                                                 int(K), _ptr(out_tri_mask), _ptr(out_normals), _ptr(out_labels),
                                                 _stream(stream)), "pl3d_extract_planes_host")


def pl3d_extract_planes_static(points, H, W, params, dominant_normals, K, out_tri_mask, out_normals, out_labels,
                               stream=None) -> int:
    """Allocation-free variant (no context; scratch in a fixed device array, frames up to
    PL3D_STATIC_MAX_POINTS points); see include/pl3d.h."""
    n_tri = 2 * (H - 1) * (W - 1)
    _check_tensor(points, "points", "torch.float32", H * W * 3)
    _check_tensor(out_tri_mask, "out_tri_mask", "torch.uint8", n_tri)
    _check_tensor(out_normals, "out_normals", "torch.float32", n_tri * 3)
    _check_tensor(out_labels, "out_labels", "torch.int32", n_tri)
    nd = _nd_host(dominant_normals, K)
    return _check(lib().pl3d_extract_planes_static(_ptr(points), int(H), int(W), ctypes.byref(params), _ptr(nd),
                                                   int(K), _ptr(out_tri_mask), _ptr(out_normals), _ptr(out_labels),
                                                   _stream(stream)), "pl3d_extract_planes_static")


def pl3d_static_scratch_bytes() -> int:
    return int(lib().pl3d_static_scratch_bytes())


PL3D_STATIC_MAX_POINTS = 307200


def pl3d_static_sync(stream=None) -> int:
    """Waits for the stream and reports a device-side timeout of the allocation-free calls."""
    return _check(lib().pl3d_static_sync(_stream(stream)), "pl3d_static_sync")


def pl3d_selftest_wait_timeout(ctx, kind: int, limit_ns: int, stream=None) -> int:
    """Makes a bounded device wait run out (kind 1: grid barrier, 2: mbarrier); ctx None targets
    the allocation-free entry point's error word. See include/pl3d.h."""
    return _check(lib().pl3d_selftest_wait_timeout(ctx or None, int(kind), int(limit_ns), _stream(stream)),
                  "pl3d_selftest_wait_timeout")


class Batch:
    """A list of frames marshalled into a C array of pl3d_frame. Keeps every buffer it points at
    (torch tensors, parameter structs, host normals) alive for as long as the batch lives."""

    def __init__(self):
        self._keep = []
        self._frames = []
        self._array = None

    def add(self, points, H, W, params, dominant_normals, out_tri_mask, out_normals, out_labels, out_points=None,
            out_groups=None):
        n_tri = 2 * (H - 1) * (W - 1)
        _check_tensor(points, "points", "torch.float32", H * W * 3)
        _check_tensor(out_tri_mask, "out_tri_mask", "torch.uint8", n_tri)
        _check_tensor(out_normals, "out_normals", "torch.float32", n_tri * 3)
        _check_tensor(out_labels, "out_labels", "torch.int32", n_tri)
        _check_tensor(out_points, "out_points", "torch.float32", H * W * 3)
        _check_tensor(out_groups, "out_groups", "torch.uint8", n_tri)
        nd = _nd_host(dominant_normals)
        p = pl3d_params(**params.as_dict()) if isinstance(params, pl3d_params) else make_params(**params)
        self._keep += [points, out_tri_mask, out_normals, out_labels, out_points, out_groups, nd, p]
        f = pl3d_frame(_ptr(points), int(H), int(W), ctypes.pointer(p), _ptr(nd), int(nd.shape[0]),
                       _ptr(out_tri_mask), _ptr(out_normals), _ptr(out_labels), _ptr(out_points), _ptr(out_groups))
        self._frames.append(f)
        self._array = None
        return len(self._frames) - 1

    def __len__(self):
        return len(self._frames)

    def array(self):
        if self._array is None:
            self._array = (pl3d_frame * max(1, len(self._frames)))(*self._frames)
        return self._array


def pl3d_extract_planes_batched(ctx, batch: Batch, stream=None) -> int:
    """All frames of `batch` in one persistent launch (a CUDA graph); see include/pl3d.h."""
    return _check(lib().pl3d_extract_planes_batched(ctx, batch.array(), len(batch), _stream(stream)),
                  "pl3d_extract_planes_batched")


def pl3d_set_tuning(ctx, tuning: Optional[pl3d_tuning] = None, **kw) -> None:
    if tuning is None and kw:
        tuning = pl3d_tuning(**kw)
    _check(lib().pl3d_set_tuning(ctx, ctypes.byref(tuning) if tuning is not None else None), "pl3d_set_tuning")


def pl3d_get_tuning(ctx) -> pl3d_tuning:
    t = pl3d_tuning()
    _check(lib().pl3d_get_tuning(ctx, ctypes.byref(t)), "pl3d_get_tuning")
    return t


def pl3d_autotune_batched(ctx, batch: Batch, stream=None, reps: int = 3):
    """Times the batch under each candidate launch shape, keeps the fastest; returns (tuning, ms)."""
    t = pl3d_tuning()
    ms = ctypes.c_double()
    _check(lib().pl3d_autotune_batched(ctx, batch.array(), len(batch), _stream(stream), int(reps), ctypes.byref(t),
                                       ctypes.byref(ms)), "pl3d_autotune_batched")
    return t, float(ms.value)


def pl3d_batch_stats(ctx) -> dict:
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().pl3d_batch_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "pl3d_batch_stats")
    return {"graph_launches": a.value, "desc_uploads": b.value, "graphs": c.value}


def pl3d_extract_mesh(ctx, points, labels, H, W, out_T, out_Tmap, out_HE, out_counts, out_seg_labels=None,
                      out_seg_offsets=None, out_seg_tris=None, out_border=None, stream=None) -> int:
    """Explicit mesh (Algorithms 1-2) and segment lists of one frame; device buffers, see include/pl3d.h."""
    n_tri = 2 * (H - 1) * (W - 1)
    _check_tensor(points, "points", "torch.float32", H * W * 3)
    _check_tensor(labels, "labels", "torch.int32", n_tri)
    _check_tensor(out_T, "out_T", "torch.int32", 3 * n_tri)
    _check_tensor(out_Tmap, "out_Tmap", "torch.int32", n_tri)
    _check_tensor(out_HE, "out_HE", "torch.int32", 3 * n_tri)
    _check_tensor(out_counts, "out_counts", "torch.int64", 3)
    _check_tensor(out_seg_labels, "out_seg_labels", "torch.int32", n_tri)
    _check_tensor(out_seg_offsets, "out_seg_offsets", "torch.int32", n_tri + 1)
    _check_tensor(out_seg_tris, "out_seg_tris", "torch.int32", n_tri)
    _check_tensor(out_border, "out_border", "torch.uint8", n_tri)
    return _check(lib().pl3d_extract_mesh(ctx, _ptr(points), _ptr(labels), int(H), int(W), _ptr(out_T), _ptr(out_Tmap),
                                          _ptr(out_HE), _ptr(out_counts), _ptr(out_seg_labels), _ptr(out_seg_offsets),
                                          _ptr(out_seg_tris), _ptr(out_border), _stream(stream)), "pl3d_extract_mesh")


def extract_mesh(ctx, points, labels, stream=None) -> dict:
    """Allocates the outputs with torch, runs pl3d_extract_mesh, waits, and returns them cut to
    their counts: T [|T|, 3], Tmap, HE [3 |T|], seg_labels, seg_offsets, seg_tris, border."""
    import torch
    H, W = int(points.shape[0]), int(points.shape[1])
    n = 2 * (H - 1) * (W - 1)
    dev = points.device
    i32 = dict(dtype=torch.int32, device=dev)
    o = dict(T=torch.empty(3 * n, **i32), Tmap=torch.empty(n, **i32), HE=torch.empty(3 * n, **i32),
             counts=torch.zeros(3, dtype=torch.int64, device=dev))
    if labels is not None:
        o.update(seg_labels=torch.empty(n, **i32), seg_offsets=torch.empty(n + 1, **i32), seg_tris=torch.empty(n, **i32),
                 border=torch.empty(n, dtype=torch.uint8, device=dev))
    pl3d_extract_mesh(ctx, points, labels, H, W, o["T"], o["Tmap"], o["HE"], o["counts"], o.get("seg_labels"),
                      o.get("seg_offsets"), o.get("seg_tris"), o.get("border"), stream)
    (torch.cuda.current_stream(dev) if stream is None else stream).synchronize()
    nT, nS, nL = (int(x) for x in o["counts"].cpu())
    out = dict(T=o["T"][:3 * nT].view(nT, 3), Tmap=o["Tmap"], HE=o["HE"][:3 * nT], counts=(nT, nS, nL))
    if labels is not None:
        out.update(seg_labels=o["seg_labels"][:nS], seg_offsets=o["seg_offsets"][:nS + 1], seg_tris=o["seg_tris"][:nL],
                   border=o["border"][:nT])
    return out


def pl3d_fastga_cells(level: int):
    """(surface normals float32 [cells, 3], 1-ring neighbours int32 [cells, 12]) of a refinement level."""
    import numpy as np
    n = 20 * 4 ** int(level)
    normals = np.empty((n, 3), np.float32)
    nbrs = np.empty((n, 12), np.int32)
    rc = lib().pl3d_fastga_cells(int(level), normals.ctypes.data, nbrs.ctypes.data)
    if rc < 0:
        raise PL3DError(rc, "pl3d_fastga_cells")
    return normals, nbrs


def pl3d_fastga(ctx, normals, mask, n, level, stride, out_counts, out_cells=None, stream=None) -> int:
    """Histogram of device normals over the cells of `level` (see include/pl3d.h)."""
    _check_tensor(normals, "normals", "torch.float32", 3 * n)
    _check_tensor(mask, "mask", "torch.uint8", n)
    _check_tensor(out_counts, "out_counts", "torch.int32", 20 * 4 ** int(level))
    _check_tensor(out_cells, "out_cells", "torch.int32", n)
    return _check(lib().pl3d_fastga(ctx, _ptr(normals), _ptr(mask), int(n), int(level), int(stride), _ptr(out_counts),
                                    _ptr(out_cells), _stream(stream)), "pl3d_fastga")


def pl3d_fastga_peaks(level, counts, v_min: float, d_peak: float, max_peaks: int = 16):
    """-> (normals float32 [p, 3], weights int64 [p]) from a host histogram."""
    import numpy as np
    c = np.ascontiguousarray(counts.cpu().numpy() if hasattr(counts, "cpu") else counts, dtype=np.int32)
    out = np.empty((max(1, max_peaks), 3), np.float32)
    w = np.empty(max(1, max_peaks), np.int64)
    k = lib().pl3d_fastga_peaks(int(level), c.ctypes.data, float(v_min), float(d_peak), int(max_peaks),
                                out.ctypes.data, w.ctypes.data)
    if k < 0:
        raise PL3DError(k, "pl3d_fastga_peaks")
    return out[:k].copy(), w[:k].copy()


def pl3d_pipeline_create(device: int = 0, max_points: int = 480 * 640, depth: int = 3) -> int:
    """A pipeline of host-buffer frames; returns its handle (see include/pl3d.h)."""
    h = _vp()
    _check(lib().pl3d_pipeline_create(int(device), int(max_points), int(depth), ctypes.byref(h)),
           "pl3d_pipeline_create")
    return int(h.value)


def pl3d_pipeline_submit(pl, points, H, W, params, dominant_normals, K, out_tri_mask, out_normals,
                         out_labels) -> int:
    """Enqueues one frame (host buffers: pinned CPU tensors that stay alive and untouched until the
    ticket is waited for); returns its ticket."""
    n_tri = 2 * (H - 1) * (W - 1)
    _check_tensor(points, "points", "torch.float32", H * W * 3, "cpu")
    _check_tensor(out_tri_mask, "out_tri_mask", "torch.uint8", n_tri, "cpu")
    _check_tensor(out_normals, "out_normals", "torch.float32", n_tri * 3, "cpu")
    _check_tensor(out_labels, "out_labels", "torch.int32", n_tri, "cpu")
    nd = _nd_host(dominant_normals, K)
    t = ctypes.c_uint64()
    _check(lib().pl3d_pipeline_submit(pl, _ptr(points), int(H), int(W), ctypes.byref(params), _ptr(nd), int(K),
                                      _ptr(out_tri_mask), _ptr(out_normals), _ptr(out_labels), ctypes.byref(t)),
           "pl3d_pipeline_submit")
    return int(t.value)


def pl3d_pipeline_wait(pl, ticket: int) -> int:
    """Waits for a frame's outputs in host memory; raises PL3DError on a failed frame."""
    return _check(lib().pl3d_pipeline_wait(pl, int(ticket)), "pl3d_pipeline_wait")


def pl3d_pipeline_status(pl, ticket: int) -> int:
    """As pl3d_pipeline_wait, returning the status code instead of raising."""
    return int(lib().pl3d_pipeline_wait(pl, int(ticket)))


def pl3d_pipeline_context(pl) -> int:
    """The pipeline's own context handle (timing, launch counts, the timeout self-test)."""
    return int(lib().pl3d_pipeline_context(pl) or 0)


def pl3d_pipeline_destroy(pl) -> None:
    lib().pl3d_pipeline_destroy(pl)


def pl3d_server_create(device: int = 0, max_inflight: int = 2, max_batch_frames: int = 64, hbm_bytes: int = 0) -> int:
    """A frame server with continuous batching; returns its handle (see include/pl3d.h)."""
    cfg = pl3d_server_config(int(device), int(max_inflight), int(max_batch_frames), 0, int(hbm_bytes))
    h = _vp()
    _check(lib().pl3d_server_create(ctypes.byref(h), ctypes.byref(cfg)), "pl3d_server_create")
    return int(h.value)


def pl3d_server_submit(srv, points, H, W, params, dominant_normals, K, out_tri_mask, out_normals, out_labels) -> int:
    """Host buffers (pinned CPU tensors or numpy arrays) that must stay alive until the ticket completes."""
    n_tri = 2 * (H - 1) * (W - 1)
    _check_tensor(points, "points", "torch.float32", H * W * 3, "cpu")
    _check_tensor(out_tri_mask, "out_tri_mask", "torch.uint8", n_tri, "cpu")
    _check_tensor(out_normals, "out_normals", "torch.float32", n_tri * 3, "cpu")
    _check_tensor(out_labels, "out_labels", "torch.int32", n_tri, "cpu")
    nd = _nd_host(dominant_normals, K)
    t = ctypes.c_uint64()
    _check(lib().pl3d_server_submit(srv, _ptr(points), int(H), int(W), ctypes.byref(params), _ptr(nd), int(K),
                                    _ptr(out_tri_mask), _ptr(out_normals), _ptr(out_labels), ctypes.byref(t)),
           "pl3d_server_submit")
    return int(t.value)


def pl3d_server_poll(srv, max_n: int = 1024, wait_ms: int = 0) -> list:
    buf = (pl3d_completion * max(1, max_n))()
    n = lib().pl3d_server_poll(srv, buf, int(max_n), int(wait_ms))
    if n < 0:
        raise PL3DError(n, "pl3d_server_poll")
    return [dict(ticket=int(c.ticket), status=int(c.status), batch_frames=int(c.batch_frames),
                 latency_ms=float(c.latency_ms), queue_ms=float(c.queue_ms)) for c in buf[:n]]


def pl3d_server_drain(srv) -> None:
    _check(lib().pl3d_server_drain(srv), "pl3d_server_drain")


def pl3d_server_get_stats(srv) -> dict:
    st = pl3d_server_stats()
    _check(lib().pl3d_server_get_stats(srv, ctypes.byref(st)), "pl3d_server_get_stats")
    return st.as_dict()


def pl3d_server_destroy(srv) -> None:
    lib().pl3d_server_destroy(srv)


def pl3d_server_replay(srv, sources: list, arrival_s, source_of) -> dict:
    """Native trace replay (see include/pl3d.h). sources: dicts with keys points (list of pinned CPU
    tensors, one per variant), params, dominant_normals, outputs (list of (mask, normals, labels)
    pinned CPU tensors, the ring). arrival_s: non-decreasing seconds; source_of: source of each
    arrival. Returns the report as a dict."""
    import numpy as np
    keep = []
    arr_src = (pl3d_replay_source * len(sources))()
    for i, sd in enumerate(sources):
        pts = sd["points"]
        H, W = int(pts[0].shape[0]), int(pts[0].shape[1])
        for t in pts:
            _check_tensor(t, "points", "torch.float32", H * W * 3, "cpu")
        n_tri = 2 * (H - 1) * (W - 1)
        for m, nrm, lab in sd["outputs"]:
            _check_tensor(m, "out_tri_mask", "torch.uint8", n_tri, "cpu")
            _check_tensor(nrm, "out_normals", "torch.float32", n_tri * 3, "cpu")
            _check_tensor(lab, "out_labels", "torch.int32", n_tri, "cpu")
        nd = _nd_host(sd["dominant_normals"])
        P = (ctypes.c_void_p * len(pts))(*[_ptr(t) for t in pts])
        M = (ctypes.c_void_p * len(sd["outputs"]))(*[_ptr(o[0]) for o in sd["outputs"]])
        N = (ctypes.c_void_p * len(sd["outputs"]))(*[_ptr(o[1]) for o in sd["outputs"]])
        L = (ctypes.c_void_p * len(sd["outputs"]))(*[_ptr(o[2]) for o in sd["outputs"]])
        prm = sd["params"]
        keep += [P, M, N, L, nd, prm]
        a = arr_src[i]
        a.host_points = ctypes.cast(P, ctypes.POINTER(ctypes.c_void_p))
        a.n_variants = len(pts)
        a.H, a.W, a.K = H, W, int(nd.shape[0])
        a.params = ctypes.pointer(prm)
        a.dominant_normals = _ptr(nd)
        a.ring = len(sd["outputs"])
        a.reserved = 0
        a.host_mask = ctypes.cast(M, ctypes.POINTER(ctypes.c_void_p))
        a.host_normals = ctypes.cast(N, ctypes.POINTER(ctypes.c_void_p))
        a.host_labels = ctypes.cast(L, ctypes.POINTER(ctypes.c_void_p))
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    which = np.ascontiguousarray(source_of, dtype=np.int32)
    rep = pl3d_replay_report()
    _check(lib().pl3d_server_replay(srv, arr_src, len(sources), _ptr(arr), _ptr(which), int(arr.shape[0]),
                                    ctypes.byref(rep)), "pl3d_server_replay")
    del keep
    return rep.as_dict()


def pl3d_sync(ctx, stream=None) -> int:
    return _check(lib().pl3d_sync(ctx, _stream(stream)), "pl3d_sync")


def pl3d_set_timing(ctx, enable: bool) -> None:
    _check(lib().pl3d_set_timing(ctx, 1 if enable else 0), "pl3d_set_timing")


def pl3d_read_timing(ctx, reset: bool = False) -> dict:
    """{phase name: (total ms, launches)} for the launches recorded while timing was on."""
    import numpy as np
    ms = np.zeros(PL3D_TIMING_SLOTS, np.float64)
    n = np.zeros(PL3D_TIMING_SLOTS, np.int64)
    rc = lib().pl3d_read_timing(ctx, ms.ctypes.data, n.ctypes.data, PL3D_TIMING_SLOTS, 1 if reset else 0)
    if rc < 0:
        raise PL3DError(rc, "pl3d_read_timing")
    return {pl3d_timing_slot_name(i): (float(ms[i]), int(n[i])) for i in range(PL3D_TIMING_SLOTS)}


def pl3d_launch_count(ctx) -> int:
    return int(lib().pl3d_launch_count(ctx))


# ----------------------------------------------------------------------------- convenience wrapper


class PlaneExtractor:
    """Owns a context and allocates outputs with torch; one call = one frame on the current stream."""

    def __init__(self, device: int = 0):
        self.device = device
        self.ctx = pl3d_create(device)

    def close(self):
        if self.ctx:
            pl3d_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __call__(self, points, params: pl3d_params, dominant_normals, want_points=False, want_groups=False,
                 stream=None):
        import torch
        H, W = int(points.shape[0]), int(points.shape[1])
        n_tri = 2 * (H - 1) * (W - 1)
        dev = points.device
        out = dict(
            mask=torch.empty(n_tri, dtype=torch.uint8, device=dev),
            normals=torch.empty((n_tri, 3), dtype=torch.float32, device=dev),
            labels=torch.empty(n_tri, dtype=torch.int32, device=dev),
        )
        if want_points:
            out["points"] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        if want_groups:
            out["groups"] = torch.empty(n_tri, dtype=torch.uint8, device=dev)
        nd = _nd_host(dominant_normals)
        pl3d_extract_planes_ex(self.ctx, points, H, W, params, nd, nd.shape[0], out["mask"], out["normals"],
                               out["labels"], out.get("points"), out.get("groups"), stream)
        return out

"""The C ABI on the CPU: the library builds, loads and exports every declared symbol; host-side
argument checks; struct layout. No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pl3d.h")


@pytest.fixture(scope="module")
def pl3d():
    from paper_2007_12065_gb300 import build
    build.build()
    import paper_2007_12065_gb300 as m
    m.lib()
    return m


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pl3d_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(pl3d):
    names = declared_functions()
    assert len(names) >= 14
    L = ctypes.CDLL(pl3d.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_every_declared_function_has_a_same_named_wrapper(pl3d):
    missing = [n for n in declared_functions() if not callable(getattr(pl3d, n, None))]
    assert not missing, missing


def test_library_is_sm103a_only(pl3d):
    from paper_2007_12065_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_struct_layout(pl3d):
    assert ctypes.sizeof(pl3d.pl3d_params) == 48
    assert pl3d.pl3d_params.min_triangles.offset == 40


def test_status_strings(pl3d):
    for code in (0, -1, -2, -3, -4, -5):
        assert pl3d.pl3d_status_string(code) != "unknown status"
    assert pl3d.pl3d_status_string(7) == "unknown status"
    assert pl3d.pl3d_version() >= 10000
    names = [pl3d.pl3d_timing_slot_name(i) for i in range(pl3d.PL3D_TIMING_SLOTS)]
    assert names == ["laplacian", "bilateral", "label_merge", "label_flatten", "frame_kernel", "host_copies",
                     "mesh_kernel", "fastga_kernel", "bil_staging_cta", "bil_geometry_cta", "bil_iterations_cta",
                     "bil_finish_cta", "bil_labels_cta"]


def test_default_params_are_paper_rgbd(pl3d):
    p = pl3d.pl3d_default_params()
    assert (p.lap_iters, p.lap_kernel, p.bil_iters, p.bil_kernel) == (2, 3, 2, 3)
    assert np.isclose(p.bil_sigma_len, 0.1) and np.isclose(p.bil_sigma_ang, 0.15)
    assert np.isclose(p.max_edge, 0.05) and np.isclose(p.min_dot, 0.96)


def test_validate(pl3d):
    nd = np.array([[0, 0, 1]], np.float32)
    ok = pl3d.make_params()
    assert pl3d.pl3d_validate(ok, 120, 160, nd) == 0
    assert pl3d.pl3d_validate(ok, 2, 2, nd) == 0
    assert pl3d.pl3d_validate(ok, 1, 160, nd) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_validate(ok, 160, 1, nd) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_validate(ok, 50000, 50000, nd) == pl3d.PL3D_ERR_INVALID_ARG     # GID overflows int32
    assert pl3d.pl3d_validate(ok, 10, 10, nd, K=0) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_validate(ok, 10, 10, None, K=255) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_validate(ok, 10, 10, None, K=254) == 0
    assert pl3d.pl3d_validate(ok, 10, 10, np.zeros((1, 3), np.float32)) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_validate(ok, 10, 10, np.array([[np.nan, 0, 1]], np.float32)) == pl3d.PL3D_ERR_INVALID_ARG
    bad = [dict(flags=1), dict(lap_iters=-1), dict(bil_iters=-1), dict(min_triangles=-1), dict(lap_lambda=1.5),
           dict(lap_lambda=-0.1), dict(lap_lambda=float("nan")), dict(bil_sigma_len=0.0),
           dict(bil_sigma_ang=float("inf")), dict(max_edge=float("nan")), dict(min_dot=float("inf")),
           dict(max_offset=float("nan"))]
    for kw in bad:
        assert pl3d.pl3d_validate(pl3d.make_params(**kw), 10, 10, nd) == pl3d.PL3D_ERR_INVALID_ARG, kw
    for kw in (dict(lap_kernel=4), dict(lap_kernel=9), dict(bil_kernel=1), dict(bil_kernel=2)):
        assert pl3d.pl3d_validate(pl3d.make_params(**kw), 10, 10, nd) == pl3d.PL3D_ERR_UNSUPPORTED, kw
    # kernel sizes are not checked for a filter that does not run
    assert pl3d.pl3d_validate(pl3d.make_params(lap_iters=0, lap_kernel=4, bil_iters=0, bil_kernel=2), 10, 10, nd) == 0


def test_binding_checks_buffers_before_the_library(pl3d):
    """The binding rejects host arrays of the wrong dtype, size or layout, host arrays handed to a
    device entry point, and K beyond the dominant normals it holds -- before any library call."""
    H, W = 4, 5
    n = 2 * (H - 1) * (W - 1)
    p = pl3d.make_params()
    nd = np.array([[0, 0, 1]], np.float32)
    pts = np.zeros((H, W, 3), np.float32)
    mask, nrm, lab = np.zeros(n, np.uint8), np.zeros((n, 3), np.float32), np.zeros(n, np.int32)
    host = pl3d.pl3d_extract_planes_host
    with pytest.raises(ValueError, match="out_labels must be int32"):
        host(0, pts, H, W, p, nd, 1, mask, nrm, lab.astype(np.int64))
    with pytest.raises(ValueError, match="out_normals must have"):
        host(0, pts, H, W, p, nd, 1, mask, nrm[:-1], lab)
    with pytest.raises(ValueError, match="points must be contiguous"):
        host(0, np.zeros((H, W, 6), np.float32)[:, :, ::2], H, W, p, nd, 1, mask, nrm, lab)
    with pytest.raises(ValueError, match="K = 2"):
        host(0, pts, H, W, p, nd, 2, mask, nrm, lab)
    with pytest.raises(ValueError, match="must be a cuda tensor"):
        pl3d.pl3d_extract_planes(0, pts, H, W, p, nd, 1, mask, nrm, lab)
    with pytest.raises(ValueError, match="K = 3"):
        pl3d.pl3d_server_submit(0, pts, H, W, p, nd, 3, mask, nrm, lab)
    assert pl3d.pl3d_validate(p, H, W, nd, K=2) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_validate(p, H, W, np.tile(nd, (2, 1)), K=2) == 0


def test_null_arguments_rejected_before_any_cuda_call(pl3d):
    L = pl3d.lib()
    p = pl3d.make_params()
    nd = np.array([[0, 0, 1]], np.float32)
    rc = L.pl3d_extract_planes(None, 1, 4, 4, ctypes.byref(p), nd.ctypes.data, 1, 1, 1, 1, None)
    assert rc == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_create(None, 0) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_sync(None, None) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_set_timing(None, 1) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_launch_count(None) == 0
    L.pl3d_destroy(None)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2007_12065_gb300 as m
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m, "LIB_PATH", str(tmp_path / "libpl3d.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        m.lib()


def test_product_path_does_not_touch_the_oracle():
    """The package and its sources never name the oracle or the scene generators."""
    pkg = os.path.join(ROOT, "paper_2007_12065_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "import synth" not in text and "from synth" not in text, f
                assert "pl3d_oracle" not in text and "liborc" not in text, f


def test_batch_and_tuning_structs(pl3d):
    assert ctypes.sizeof(pl3d.pl3d_frame) == 80
    assert pl3d.pl3d_frame.params.offset == 16 and pl3d.pl3d_frame.K.offset == 32
    assert pl3d.pl3d_frame.out_groups.offset == 72
    assert ctypes.sizeof(pl3d.pl3d_tuning) == 20 and pl3d.pl3d_tuning.bil_tile_h.offset == 16


def test_batch_and_tuning_null_arguments(pl3d):
    L = pl3d.lib()
    t = pl3d.pl3d_tuning(1, 1, 1)
    assert L.pl3d_extract_planes_batched(None, None, 0, None) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_set_tuning(None, ctypes.byref(t)) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_get_tuning(None, ctypes.byref(t)) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_autotune_batched(None, None, 1, None, 3, None, None) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_batch_stats(None, None, None, None) == pl3d.PL3D_ERR_INVALID_ARG


def test_server_structs_and_config_checks(pl3d):
    assert ctypes.sizeof(pl3d.pl3d_server_config) == 24
    assert ctypes.sizeof(pl3d.pl3d_completion) == 32
    assert ctypes.sizeof(pl3d.pl3d_server_stats) == 64
    L = pl3d.lib()
    h = ctypes.c_void_p()
    for cfg in [(0, 0, 8, 0, 0), (0, 3, 8, 0, 0), (0, 1, 0, 0, 0), (0, 1, 5000, 0, 0), (0, 1, 8, 1, 0),
                (0, 1, 8, 0, -1)]:
        c = pl3d.pl3d_server_config(*cfg)
        assert L.pl3d_server_create(ctypes.byref(h), ctypes.byref(c)) == pl3d.PL3D_ERR_INVALID_ARG, cfg
    assert L.pl3d_server_create(None, None) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_server_submit(None, None, 4, 4, None, None, 1, None, None, None, None) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_server_poll(None, None, 0, 0) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_server_drain(None) == pl3d.PL3D_ERR_INVALID_ARG
    assert L.pl3d_server_get_stats(None, None) == pl3d.PL3D_ERR_INVALID_ARG
    L.pl3d_server_destroy(None)


def test_static_entry_point_limits_before_any_cuda_call(pl3d):
    """The allocation-free call refuses what its fixed scratch cannot hold -- frames above
    640 x 480 points, more than one bilateral pass, the host-assisted seeded mode -- on the host,
    before it touches the device (the device pointers here are placeholders never dereferenced)."""
    L = pl3d.lib()
    nd = np.array([[0, 0, 1]], np.float32)
    dummy = 256

    def call(H, W, **kw):
        p = pl3d.make_params(**kw)
        return L.pl3d_extract_planes_static(dummy, H, W, ctypes.byref(p), nd.ctypes.data, 1, dummy, dummy, dummy,
                                            None)
    assert call(481, 640) == pl3d.PL3D_ERR_INVALID_ARG          # 307,840 points > 307,200
    assert call(640, 481) == pl3d.PL3D_ERR_INVALID_ARG
    assert call(120, 160, bil_iters=12) == pl3d.PL3D_ERR_INVALID_ARG   # halo 12 > 6 quads: two passes
    assert call(120, 160, flags=pl3d.PL3D_FLAG_SEED_PTP, max_offset=0.1) == pl3d.PL3D_ERR_UNSUPPORTED
    assert call(1, 160) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.pl3d_static_scratch_bytes() >= 307200 * 24

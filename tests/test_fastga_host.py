"""The library's Gaussian-accumulator tables and host peak detector against the oracle (CPU only:
these entry points make no CUDA call)."""
import numpy as np
import pytest

from oracle import fastga


@pytest.fixture(scope="module")
def pl3d():
    from paper_2007_12065_gb300 import build
    build.build()
    import paper_2007_12065_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_cell_tables_match_oracle(pl3d, level):
    normals, nbrs = pl3d.pl3d_fastga_cells(level)
    V, F = fastga.icosahedron(level)
    N = fastga.cell_normals(V, F)
    assert normals.shape == N.shape
    assert np.abs(normals - N).max() < 1e-7                      # FP32 rounding of the same normals
    ref = fastga.neighbours(F)
    for i in range(0, len(F), max(1, len(F) // 2000)):
        row = [int(x) for x in nbrs[i] if x >= 0]
        assert row == ref[i], i
        assert all(x == -1 for x in nbrs[i][len(row):])


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_search_tables_pass_their_check(pl3d, level):
    """The device search treats every level-0 face as a rotated copy of face 0; the library checks
    on the host, for every cell of face 0's neighbourhood, that the rotation lands on a cell normal
    with the same child number, and reports a failure from pl3d_fastga_cells."""
    assert pl3d.lib().pl3d_fastga_cells(level, None, None) == 20 * 4 ** level


def test_invalid_level_rejected(pl3d):
    assert pl3d.lib().pl3d_fastga_cells(6, None, None) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.lib().pl3d_fastga_cells(-1, None, None) == pl3d.PL3D_ERR_INVALID_ARG
    assert pl3d.lib().pl3d_fastga(None, None, None, 0, 3, 1, None, None, None) == pl3d.PL3D_ERR_INVALID_ARG


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_peaks_match_oracle(pl3d, seed):
    level = 3
    V, F = fastga.icosahedron(level)
    N = fastga.cell_normals(V, F)
    rng = np.random.default_rng(seed)
    counts = rng.poisson(3.0, len(F)).astype(np.int64)
    for _ in range(6):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        counts += np.round(rng.uniform(100, 900) * np.exp(-(1 - N @ d) / 4e-3)).astype(np.int64)
    for d_peak in (0.05, 0.3, 0.8):
        ref_n, ref_w = fastga.peaks(counts, level, v_min=20.0, d_peak=d_peak)
        got_n, got_w = pl3d.pl3d_fastga_peaks(level, counts.astype(np.int32), 20.0, d_peak, max_peaks=64)
        assert np.array_equal(got_w, ref_w)
        assert np.abs(got_n - ref_n).max() < 1e-6


def test_peaks_plateau_and_threshold_match_oracle(pl3d):
    """The conventions the random histograms rarely meet: a two-cell plateau (one peak, the lower
    index) and a count equal to v_min (no peak)."""
    level = 2
    V, F = fastga.icosahedron(level)
    nb = fastga.neighbours(F)
    a = 37
    cases = []
    c = np.zeros(len(F), np.int64)
    c[a] = c[max(nb[a])] = 50
    cases.append((c, 10.0))
    c = np.zeros(len(F), np.int64)
    c[a] = 20
    cases += [(c, 20.0), (c, 19.0)]
    for counts, v_min in cases:
        ref_n, ref_w = fastga.peaks(counts, level, v_min=v_min, d_peak=0.01)
        got_n, got_w = pl3d.pl3d_fastga_peaks(level, counts.astype(np.int32), v_min, 0.01, max_peaks=8)
        assert np.array_equal(got_w, ref_w)
        assert got_n.shape == ref_n.shape and (got_n.size == 0 or np.abs(got_n - ref_n).max() < 1e-6)

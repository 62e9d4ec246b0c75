"""The pins catch plausible mistakes: each case plants one slip in a temporary copy of the oracle's C
source, of its Python layer (pipeline, near-threshold flags, segment lists and borders) or of its
Gaussian-accumulator module (on the CPU), and requires the pin suite to fail against it."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "widen_nan_in_x_only": ("if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {", "if (!isnan(p[0])) {"),
    "widen_keeps_inf": ("if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {",
                        "if (!isnan(p[0]) && !isnan(p[1]) && !isnan(p[2])) {"),
    "laplacian_sign": ("vo[0] = vi[0] + j0 * (lambda * sx / wsum);", "vo[0] = vi[0] - j0 * (lambda * sx / wsum);"),
    "laplacian_weight": ("double w = 1.0 / d; /* Eq. 2 */", "double w = 1.0 / (d * d);"),
    "laplacian_border": ("int border = (u < r) || (u >= H - r) || (v < r) || (v >= W - r);",
                         "int border = (u < r) || (u >= H - r) || (v < r);"),
    "bilateral_excludes_self": ("if (isnan(nj[0]) || isnan(cj[0])) continue;",
                                "if (isnan(nj[0]) || isnan(cj[0]) || j == i) continue;"),
    "bilateral_one_triangle_per_quad": ("for (int kk = 0; kk < 2; ++kk) {", "for (int kk = 0; kk < 1; ++kk) {"),
    "bilateral_sigma_squared": ("const double two_sc2 = 2.0 * sigma_c * sigma_c;",
                                "const double two_sc2 = sigma_c * sigma_c;"),
    "bilateral_no_normal_term": ("double w = wc * ws;", "double w = wc;"),
    "bilateral_no_renormalisation": ("no[0] = sx / len;", "no[0] = sx;"),
    "vertex_order": ("        idx[0] = p3;\n        idx[1] = p2;", "        idx[0] = p2;\n        idx[1] = p3;"),
    "centroid": ("cc[2] = (a[2] + b[2] + c[2]) / 3.0;", "cc[2] = (a[2] + b[2]) / 2.0;"),
    "classify_last_wins_ties": ("if (s > max_similarity) {", "if (s >= max_similarity) {"),
    "classify_rejects_equal": ("if (max_similarity < ang_min) g = 255;", "if (max_similarity <= ang_min) g = 255;"),
    "mask_rejects_equal": ("mask[gid] = (l_max <= 0.0 || !(longest > l_max)) ? 1 : 0;",
                           "mask[gid] = (l_max <= 0.0 || longest < l_max) ? 1 : 0;"),
    "twin_top_wrong_triangle": ("if (u - 1 >= 0) out[n++] = 2 * ((int64_t)(u - 1) * Wq + v) + 1;",
                                "if (u - 1 >= 0) out[n++] = 2 * ((int64_t)(u - 1) * Wq + v);"),
    "twin_right_wrong_triangle": ("if (v + 1 < Wq) out[n++] = 2 * ((int64_t)u * Wq + v + 1) + 1;",
                                  "if (v + 1 < Wq) out[n++] = 2 * ((int64_t)u * Wq + v + 1);"),
    "tri_min_not_strict": ("if (tri_min > 0 && tail <= (int64_t)tri_min) {",
                           "if (tri_min > 0 && tail < (int64_t)tri_min) {"),
    "halfedge_top_wrong_edge": ("if (top != -1) HE[3 * (int64_t)first + 1] = 3 * top + 1;",
                                "if (top != -1) HE[3 * (int64_t)first + 1] = 3 * top;"),
    "laplacian_nan_neighbour_used": ("                        if (isnan(vj[0])) continue;\n", ""),
    "laplacian_zero_distance_used": ("                        if (d == 0.0) continue;\n", ""),
    "laplacian_border_width_one": ("int border = (u < r) || (u >= H - r) || (v < r) || (v >= W - r);",
                                   "int border = (u < 1) || (u >= H - 1) || (v < 1) || (v >= W - 1);"),
    "laplacian_lambda_dropped": ("vo[1] = vi[1] + j1 * (lambda * sy / wsum);", "vo[1] = vi[1] + j1 * (sy / wsum);"),
    "laplacian_in_place_sweep": ("const double* vj = cur + 3 * ((size_t)(u + du) * W + (v + dv));",
                                 "const double* vj = (du < 0 || (du == 0 && dv < 0) ? nxt : cur) + "
                                 "3 * ((size_t)(u + du) * W + (v + dv));"),
    "bilateral_centroid_term_uses_sigma_s": ("exp(-(dcx * dcx + dcy * dcy + dcz * dcz) / two_sc2)",
                                             "exp(-(dcx * dcx + dcy * dcy + dcz * dcz) / two_ss2)"),
    "bilateral_border_replicated": ("                        int uu = u + du;\n                        if (uu < 0 || uu >= Hq) continue;",
                                    "                        int uu = u + du;\n                        uu = uu < 0 ? 0 : (uu >= Hq ? Hq - 1 : uu);"),
    "bilateral_in_place_sweep": ("const double* nj = cur + 3 * j;", "const double* nj = (j < i ? nxt : cur) + 3 * j;"),
    "degenerate_threshold_zero": ("if (!(len > 1e-20)) {", "if (!(len > 0.0)) {"),
    "normal_not_unit": ("                nn[0] = nx / len;\n", "                nn[0] = nx;\n"),
    "classify_unsigned_dot": ("double s = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];\n                if (s > max_similarity) {",
                              "double s = fabs(n[0] * d[0] + n[1] * d[1] + n[2] * d[2]);\n"
                              "                if (s > max_similarity) {"),
    "offset_test_signed": ("if (fabs(off) > max_offset) continue;", "if (off > max_offset) continue;"),
    "offset_drops_y_term": ("double off = d[0] * (ct[0] - cj[0]) + d[1] * (ct[1] - cj[1]) +",
                            "double off = d[0] * (ct[0] - cj[0]) + d[1] * (ct[1] - ct[1]) +"),
    "label_ignores_group": ("if (labels[j] != UNVISITED || G[j] != g) continue;\n                if (max_offset > 0.0 && g < K) {",
                            "if (labels[j] != UNVISITED) continue;\n                if (max_offset > 0.0 && g < K) {"),
    "label_seeds_reversed": ("const int32_t UNVISITED = -2;\n    for (int64_t t = 0; t < n; ++t) labels[t] = (G[t] == 255) ? -1 : "
                             "UNVISITED;\n    for (int64_t seed = 0; seed < n; ++seed) {",
                             "const int32_t UNVISITED = -2;\n    for (int64_t t = 0; t < n; ++t) labels[t] = (G[t] == 255) ? -1 : "
                             "UNVISITED;\n    for (int64_t seed = n - 1; seed >= 0; --seed) {"),
    "mask_edges_on_raw_points": ("const double* a = P_smooth + 3 * idx[m];\n                    const double* b = P_smooth + 3 * idx[(m + 1) % 3];",
                                 "const double* a = P_raw + 3 * idx[m];\n                    const double* b = P_raw + 3 * idx[(m + 1) % 3];"),
    "mask_two_edges_only": ("                for (int m = 0; m < 3; ++m) {\n                    const double* a = P_smooth",
                            "                for (int m = 0; m < 2; ++m) {\n                    const double* a = P_smooth"),
    "extract_misses_third_vertex": ("if (isnan(P_raw[3 * idx[0]]) || isnan(P_raw[3 * idx[1]]) ||\n                    isnan(P_raw[3 * idx[2]])) {",
                                    "if (isnan(P_raw[3 * idx[0]]) || isnan(P_raw[3 * idx[1]])) {"),
    "halfedge_bottom_wrong_edge": ("if (bottom != -1) HE[3 * (int64_t)second + 1] = 3 * bottom + 1;",
                                   "if (bottom != -1) HE[3 * (int64_t)second + 1] = 3 * bottom;"),
    "halfedge_left_wrong_triangle": ("int32_t left = (v - 1 >= 0) ? Tmap[2 * ((int64_t)u * Wq + v - 1)] : -1;",
                                     "int32_t left = (v - 1 >= 0) ? Tmap[2 * ((int64_t)u * Wq + v - 1) + 1] : -1;"),
    "seeded_dropped_triangles_released": (
        "if (tri_min > 0 && tail <= (int64_t)tri_min)\n            for (int64_t a = 0; a < tail; ++a) labels[queue[a]] = -1;",
        "if (tri_min > 0 && tail <= (int64_t)tri_min)\n            for (int64_t a = 0; a < tail; ++a) "
        "labels[queue[a]] = a == 0 ? -1 : UNVISITED;"),
    "seeded_tri_min_not_strict": ("if (tri_min > 0 && tail <= (int64_t)tri_min)\n            for",
                                  "if (tri_min > 0 && tail < (int64_t)tri_min)\n            for"),
    "seeded_offset_from_previous_triangle": (
        "fabs(d[0] * (cj[0] - cs[0]) + d[1] * (cj[1] - cs[1]) + d[2] * (cj[2] - cs[2]))",
        "fabs(d[0] * (cj[0] - C[3 * t]) + d[1] * (cj[1] - C[3 * t + 1]) + d[2] * (cj[2] - C[3 * t + 2]))"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "pl3d_oracle.c")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    (tmp_path / "oracle" / "pl3d_oracle.c").write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x", "-p", "no:cacheprovider"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and "failed" in r.stdout, r.stdout[-2000:]


FASTGA_MUTATIONS = {
    "child_order_swapped": ("nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]",
                            "nxt += [(ab, b, bc), (a, ab, ca), (ca, bc, c), (ab, bc, ca)]"),
    "centre_child_reversed": ("nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]",
                              "nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, ca, bc)]"),
    "midpoint_not_projected": ("V.append(p / np.linalg.norm(p))", "V.append(p / 2.0)"),
    "cell_normals_not_unit": ("return n / np.linalg.norm(n, axis=1)[:, None]", "return n"),
    "nearest_smallest_dot": ("out[s:s + chunk] = (normals[s:s + chunk] @ N.T).argmax(1)",
                             "out[s:s + chunk] = (normals[s:s + chunk] @ N.T).argmin(1)"),
    "sampling_offset": ("idx = np.arange(0, len(normals), stride)", "idx = np.arange(stride - 1, len(normals), stride)"),
    "mask_ignored": ("ok &= np.asarray(mask).reshape(-1)[idx] != 0", "ok &= np.asarray(mask).reshape(-1)[idx] >= 0"),
    "plateau_keeps_highest_index": ("(counts[i] == counts[j] and i < j)", "(counts[i] == counts[j] and i > j)"),
    "plateau_drops_all": ("counts[i] > counts[j] or (counts[i] == counts[j] and i < j) for j in nb[i])",
                          "counts[i] > counts[j] for j in nb[i])"),
    "v_min_not_strict": ("counts[i] > v_min and all(", "counts[i] >= v_min and all("),
    "merge_unweighted": ("w = counts[members].astype(np.float64)", "w = np.ones(len(members))"),
}


@pytest.mark.parametrize("name", sorted(FASTGA_MUTATIONS))
def test_planted_fastga_mistake_fails_a_pin(name, tmp_path):
    old, new = FASTGA_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "fastga.py")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    for d in ("oracle", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    (tmp_path / "oracle" / "fastga.py").write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_fastga.py", "-q", "-x", "-p", "no:cacheprovider"],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and "failed" in r.stdout, r.stdout[-2000:]


PY_MUTATIONS = {
    "pipeline_mask_on_raw": ("m, edge = mask(raw, smoothed, p.max_edge)", "m, edge = mask(raw, raw, p.max_edge)"),
    "pipeline_smoothing_skipped": ("smoothed = laplacian(raw, p.lap_kernel, p.lap_lambda, p.lap_iters)\n",
                                   "smoothed = raw\n"),
    "border_labels_by_t_index": ("T_labels = np.asarray(labels)[gid_of]", "T_labels = np.asarray(labels)[:len(T)]"),
    "border_ignores_other_label": ("border = (T_labels >= 0) & ((tw < 0) | (other != T_labels))",
                                   "border = (T_labels >= 0) & (tw < 0)"),
    "border_on_unlabelled": ("border = (T_labels >= 0) & ((tw < 0) | (other != T_labels))",
                             "border = (tw < 0) | (other != T_labels)"),
    "segment_lists_gids_not_t": ("Tmap[gids[order]].astype(np.int32)", "gids[order].astype(np.int32)"),
    "segment_lists_not_by_label": ('order = np.argsort(lab, kind="stable")', "order = np.arange(len(lab))"),
    "near_edge_wider": ("< NEAR) & (p.max_edge > 0)", "< 10 * NEAR) & (p.max_edge > 0)"),
    "near_tie_reversed": ("((np.where(has_second, best - second, 1.0)) < NEAR)",
                          "((np.where(has_second, second - best, 1.0)) < NEAR)"),
    "near_dot_wider": ("near_dot = has_best & (np.abs(np.where(has_best, best, 0.0) - p.min_dot) < NEAR)",
                       "near_dot = has_best & (np.abs(np.where(has_best, best, 0.0) - p.min_dot) < 1e-3)"),
}


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_planted_pipeline_mistake_fails_a_pin(name, tmp_path):
    old, new = PY_MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    (tmp_path / "oracle" / "__init__.py").write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "tests/test_compare_host.py", "-q",
                        "-x", "-p", "no:cacheprovider"], cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and "failed" in r.stdout, r.stdout[-2000:]

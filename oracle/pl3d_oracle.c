/*
 * pl3d_oracle.c -- plain, slow, FP64 CPU oracle for the organized-point-cloud
 * plane-extraction path of Polylidar3D (Castagno & Atkins, arXiv 2007.12065).
 *
 * TEST INFRASTRUCTURE. This file exists only to check the CUDA path. It shares
 * no code, header, table or constant with the library under
 * paper_2007_12065_gb300/, and only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it. Nothing in the product path calls
 * it.
 *
 * Every step follows the paper's definition in the paper's order, written as
 * straightforward loops in double precision:
 *
 *   orc_widen             organized cloud, invalid points = NaN      (Section 3, Section 4.2)
 *   orc_laplacian         Laplacian vertex filter, Jacobi iterations (Eq. 1-2, Section 5.1)
 *   orc_triangle_geometry centroids and unit normals over T_FC       (Section 4.2, Algorithm 1, Section 5.2)
 *   orc_mask              triangle validity and edge-length predicate (Algorithm 1, Algorithm 4)
 *   orc_bilateral         bilateral normal filter, Jacobi iterations (Eq. 3-6, Section 5.2)
 *   orc_classify          group assignment                           (Algorithm 4)
 *   orc_label             edge-connected region growing per group    (Algorithm 5 over Algorithm 2 twins)
 *   orc_label_seeded      region growing with the seed-relative point-to-plane limit (Algorithm 5)
 *   orc_extract_triangles explicit triangle set T and map T_map      (Algorithm 1)
 *   orc_extract_halfedges explicit twin array HE                     (Algorithm 2)
 *
 * Readings taken where the paper is silent or garbled, each with the reason
 * it is taken:
 *   - Eq. 1 prints a product and an outward sign; the standard umbrella form
 *     v' = v + (lambda / W) * sum_j w_j (v_j - v) is used (Taubin, cited there).
 *   - Laplacian neighbours: the k x k image window minus the vertex itself,
 *     invalid (NaN) neighbours and neighbours at distance exactly 0 skipped;
 *     W = 0 leaves the vertex unchanged; the ring of width floor(k/2) at the
 *     image border is not filtered (Section 5.1).
 *   - Both filters are Jacobi (every iteration reads the previous one only).
 *   - Bilateral window: both triangles of every quad in the k x k quad window
 *     centred on the triangle's quad, the triangle itself included; NaN and
 *     out-of-image triangles skipped; the weighted sum is renormalised to unit
 *     length each iteration (the factor K of Eq. 3 cancels there); centroids
 *     stay fixed; a triangle whose normal is NaN stays NaN.
 *   - sigma_c and sigma_s are standard deviations: exp(-d^2 / (2 sigma^2)).
 *   - A triangle whose cross product has length <= 1e-20 has no normal (NaN);
 *     its centroid stays defined.
 *   - The edge-length predicate of Algorithm 4 uses the smoothed vertices and
 *     rejects only when the longest edge is strictly greater than l_max.
 *   - Group assignment uses signed dot products, strict '>' (lowest index wins
 *     ties), and rejects when the best dot is strictly below ang_min.
 *   - Region growing is order independent: a component is every triangle
 *     reachable through twin half-edges with the same group (and, when
 *     max_offset > 0, |n^d_g . (c_i - c_j)| <= max_offset between the two
 *     triangles). Its label is its smallest GID. Components of at most tri_min
 *     triangles are dropped when tri_min > 0 (Algorithm 5 keeps |T^g_i| > tri_min).
 *   - No wrap between the last and the first image column.
 *
 * Sensitivity runs (test instrumentation, not part of the method): orc_laplacian_jitter and
 * orc_bilateral_jitter repeat the filters with every update scaled by (1 + eps r), r = +-1
 * drawn from a counter-based hash (SplitMix64 finaliser) of (seed, iteration, index,
 * coordinate). With eps of the order of FP32 rounding (2^-22) they show which outputs the
 * problem itself does not determine to FP32 precision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

static int g_threads = 1;

/* SplitMix64 finaliser (Steele, Lea, Flood 2014) used as a counter-based hash. */
static uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* +1 or -1 from (seed, iteration, index, coordinate). */
static double jitter_sign(uint64_t seed, int it, int64_t index, int comp) {
    uint64_t h = mix64(seed ^ mix64(((uint64_t)it << 48) ^ ((uint64_t)index << 2) ^ (uint64_t)comp));
    return (h >> 63) ? 1.0 : -1.0;
}

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int orc_get_threads(void) { return g_threads; }

int orc_has_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* ------------------------------------------------------------------------ */
/* Section 3 / Section 4.2: an organized cloud keeps its grid; an invalid     */
/* point (any non-finite coordinate) becomes NaN in all three coordinates.   */
/* ------------------------------------------------------------------------ */
void orc_widen(const float* pts, int64_t n_points, double* out) {
    for (int64_t i = 0; i < n_points; ++i) {
        const float* p = pts + 3 * i;
        double* o = out + 3 * i;
        if (isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2])) {
            o[0] = (double)p[0];
            o[1] = (double)p[1];
            o[2] = (double)p[2];
        } else {
            o[0] = NAN;
            o[1] = NAN;
            o[2] = NAN;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. 1-2, Section 5.1: Laplacian filter on the implicit grid.              */
/* ------------------------------------------------------------------------ */
int orc_laplacian_jitter(const double* P0, int H, int W, int kernel, double lambda, int iters,
                         double eps, uint64_t seed, double* out) {
    if (H < 1 || W < 1 || kernel < 1 || (kernel % 2) == 0 || iters < 0) return ORC_EINVAL;
    const int r = kernel / 2;
    const size_t n = (size_t)H * (size_t)W * 3u;
    double* cur = (double*)malloc(n * sizeof(double));
    double* nxt = (double*)malloc(n * sizeof(double));
    if (!cur || !nxt) {
        free(cur);
        free(nxt);
        return ORC_ENOMEM;
    }
    memcpy(cur, P0, n * sizeof(double));
    for (int it = 0; it < iters; ++it) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
        for (int u = 0; u < H; ++u) {
            for (int v = 0; v < W; ++v) {
                const double* vi = cur + 3 * ((size_t)u * W + v);
                double* vo = nxt + 3 * ((size_t)u * W + v);
                int border = (u < r) || (u >= H - r) || (v < r) || (v >= W - r);
                if (isnan(vi[0]) || border) {
                    vo[0] = vi[0];
                    vo[1] = vi[1];
                    vo[2] = vi[2];
                    continue;
                }
                double sx = 0.0, sy = 0.0, sz = 0.0, wsum = 0.0;
                for (int du = -r; du <= r; ++du) {
                    for (int dv = -r; dv <= r; ++dv) {
                        if (du == 0 && dv == 0) continue;
                        const double* vj = cur + 3 * ((size_t)(u + du) * W + (v + dv));
                        if (isnan(vj[0])) continue;
                        double dx = vj[0] - vi[0], dy = vj[1] - vi[1], dz = vj[2] - vi[2];
                        double d = sqrt(dx * dx + dy * dy + dz * dz);
                        if (d == 0.0) continue;
                        double w = 1.0 / d; /* Eq. 2 */
                        sx += w * dx;
                        sy += w * dy;
                        sz += w * dz;
                        wsum += w;
                    }
                }
                if (wsum > 0.0) {
                    double j0 = 1.0, j1 = 1.0, j2 = 1.0;
                    if (eps != 0.0) {
                        int64_t pi = (int64_t)u * W + v;
                        j0 += eps * jitter_sign(seed, it, pi, 0);
                        j1 += eps * jitter_sign(seed, it, pi, 1);
                        j2 += eps * jitter_sign(seed, it, pi, 2);
                    }
                    vo[0] = vi[0] + j0 * (lambda * sx / wsum); /* Eq. 1, umbrella form */
                    vo[1] = vi[1] + j1 * (lambda * sy / wsum);
                    vo[2] = vi[2] + j2 * (lambda * sz / wsum);
                } else {
                    vo[0] = vi[0];
                    vo[1] = vi[1];
                    vo[2] = vi[2];
                }
            }
        }
        double* t = cur;
        cur = nxt;
        nxt = t;
    }
    memcpy(out, cur, n * sizeof(double));
    free(cur);
    free(nxt);
    return ORC_OK;
}

int orc_laplacian(const double* P0, int H, int W, int kernel, double lambda, int iters, double* out) {
    return orc_laplacian_jitter(P0, H, W, kernel, lambda, iters, 0.0, 0, out);
}

/* ------------------------------------------------------------------------ */
/* Section 4.2 / Algorithm 1: the vertices of triangle (u, v, k) of T_FC.    */
/* Quad (u, v): p1 = (u, v), p2 = (u, v+1), p3 = (u+1, v+1), p4 = (u+1, v).  */
/* First (k = 0) = {p3, p2, p1}; second (k = 1) = {p1, p4, p3}.              */
/* GID = 2 (u (W-1) + v) + k.                                                */
/* ------------------------------------------------------------------------ */
static void tri_vertex_index(int u, int v, int k, int W, int64_t idx[3]) {
    int64_t p1 = (int64_t)u * W + v;
    int64_t p2 = (int64_t)u * W + v + 1;
    int64_t p3 = (int64_t)(u + 1) * W + v + 1;
    int64_t p4 = (int64_t)(u + 1) * W + v;
    if (k == 0) {
        idx[0] = p3;
        idx[1] = p2;
        idx[2] = p1;
    } else {
        idx[0] = p1;
        idx[1] = p4;
        idx[2] = p3;
    }
}

/* Section 5.2: centroid and unit normal of every triangle of T_FC (NaN when a
 * vertex is NaN). The normal follows the right-hand rule over the listed
 * vertex order: n = (b - a) x (c - a) / |(b - a) x (c - a)|. */
int orc_triangle_geometry(const double* P, int H, int W, double* C, double* N) {
    if (H < 2 || W < 2) return ORC_EINVAL;
    const int Wq = W - 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (int u = 0; u < H - 1; ++u) {
        for (int v = 0; v < Wq; ++v) {
            for (int k = 0; k < 2; ++k) {
                int64_t gid = 2 * ((int64_t)u * Wq + v) + k;
                int64_t idx[3];
                tri_vertex_index(u, v, k, W, idx);
                const double* a = P + 3 * idx[0];
                const double* b = P + 3 * idx[1];
                const double* c = P + 3 * idx[2];
                double* cc = C + 3 * gid;
                double* nn = N + 3 * gid;
                if (isnan(a[0]) || isnan(b[0]) || isnan(c[0])) {
                    cc[0] = cc[1] = cc[2] = NAN;
                    nn[0] = nn[1] = nn[2] = NAN;
                    continue;
                }
                cc[0] = (a[0] + b[0] + c[0]) / 3.0;
                cc[1] = (a[1] + b[1] + c[1]) / 3.0;
                cc[2] = (a[2] + b[2] + c[2]) / 3.0;
                double e1x = b[0] - a[0], e1y = b[1] - a[1], e1z = b[2] - a[2];
                double e2x = c[0] - a[0], e2y = c[1] - a[1], e2z = c[2] - a[2];
                double nx = e1y * e2z - e1z * e2y;
                double ny = e1z * e2x - e1x * e2z;
                double nz = e1x * e2y - e1y * e2x;
                double len = sqrt(nx * nx + ny * ny + nz * nz);
                if (!(len > 1e-20)) {
                    nn[0] = nn[1] = nn[2] = NAN;
                    continue;
                }
                nn[0] = nx / len;
                nn[1] = ny / len;
                nn[2] = nz / len;
            }
        }
    }
    return ORC_OK;
}

/* Algorithm 1 (all three vertices valid in the raw cloud) and the first
 * predicate of Algorithm 4 (longest edge, on the smoothed vertices, not
 * greater than l_max; l_max <= 0 disables the predicate). max_edge_len gets
 * the longest edge (NaN for triangles with an invalid vertex). */
int orc_mask(const double* P_raw, const double* P_smooth, int H, int W, double l_max,
             uint8_t* mask, double* max_edge_len) {
    if (H < 2 || W < 2) return ORC_EINVAL;
    const int Wq = W - 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (int u = 0; u < H - 1; ++u) {
        for (int v = 0; v < Wq; ++v) {
            for (int k = 0; k < 2; ++k) {
                int64_t gid = 2 * ((int64_t)u * Wq + v) + k;
                int64_t idx[3];
                tri_vertex_index(u, v, k, W, idx);
                int valid = 1;
                for (int m = 0; m < 3; ++m)
                    if (isnan(P_raw[3 * idx[m]])) valid = 0;
                if (!valid) {
                    mask[gid] = 0;
                    if (max_edge_len) max_edge_len[gid] = NAN;
                    continue;
                }
                double longest = 0.0;
                for (int m = 0; m < 3; ++m) {
                    const double* a = P_smooth + 3 * idx[m];
                    const double* b = P_smooth + 3 * idx[(m + 1) % 3];
                    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
                    double len = sqrt(dx * dx + dy * dy + dz * dz);
                    if (len > longest) longest = len;
                }
                if (max_edge_len) max_edge_len[gid] = longest;
                mask[gid] = (l_max <= 0.0 || !(longest > l_max)) ? 1 : 0;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3-6, Section 5.2: bilateral filter of triangle normals over T_FC.     */
/* ------------------------------------------------------------------------ */
int orc_bilateral_jitter(const double* C, const double* N0, int H, int W, int kernel, double sigma_c,
                         double sigma_s, int iters, double eps, uint64_t seed, double* Nout) {
    if (H < 2 || W < 2 || kernel < 1 || (kernel % 2) == 0 || iters < 0) return ORC_EINVAL;
    if (!(sigma_c > 0.0) || !(sigma_s > 0.0)) return ORC_EINVAL;
    const int r = kernel / 2;
    const int Hq = H - 1, Wq = W - 1;
    const size_t n = (size_t)Hq * (size_t)Wq * 2u * 3u;
    double* cur = (double*)malloc(n * sizeof(double));
    double* nxt = (double*)malloc(n * sizeof(double));
    if (!cur || !nxt) {
        free(cur);
        free(nxt);
        return ORC_ENOMEM;
    }
    memcpy(cur, N0, n * sizeof(double));
    const double two_sc2 = 2.0 * sigma_c * sigma_c;
    const double two_ss2 = 2.0 * sigma_s * sigma_s;
    for (int it = 0; it < iters; ++it) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
        for (int u = 0; u < Hq; ++u) {
            for (int v = 0; v < Wq; ++v) {
                for (int k = 0; k < 2; ++k) {
                    int64_t i = 2 * ((int64_t)u * Wq + v) + k;
                    const double* ni = cur + 3 * i;
                    const double* ci = C + 3 * i;
                    double* no = nxt + 3 * i;
                    if (isnan(ni[0])) {
                        no[0] = no[1] = no[2] = NAN;
                        continue;
                    }
                    double sx = 0.0, sy = 0.0, sz = 0.0;
                    for (int du = -r; du <= r; ++du) {
                        int uu = u + du;
                        if (uu < 0 || uu >= Hq) continue;
                        for (int dv = -r; dv <= r; ++dv) {
                            int vv = v + dv;
                            if (vv < 0 || vv >= Wq) continue;
                            for (int kk = 0; kk < 2; ++kk) {
                                int64_t j = 2 * ((int64_t)uu * Wq + vv) + kk;
                                const double* nj = cur + 3 * j;
                                const double* cj = C + 3 * j;
                                if (isnan(nj[0]) || isnan(cj[0])) continue;
                                double dcx = ci[0] - cj[0], dcy = ci[1] - cj[1],
                                       dcz = ci[2] - cj[2];
                                double dnx = ni[0] - nj[0], dny = ni[1] - nj[1],
                                       dnz = ni[2] - nj[2];
                                double wc = exp(-(dcx * dcx + dcy * dcy + dcz * dcz) / two_sc2); /* Eq. 4 */
                                double ws = exp(-(dnx * dnx + dny * dny + dnz * dnz) / two_ss2); /* Eq. 5 */
                                double w = wc * ws;
                                sx += w * nj[0];
                                sy += w * nj[1];
                                sz += w * nj[2];
                            }
                        }
                    }
                    if (eps != 0.0) {
                        sx *= 1.0 + eps * jitter_sign(seed, it, i, 0);
                        sy *= 1.0 + eps * jitter_sign(seed, it, i, 1);
                        sz *= 1.0 + eps * jitter_sign(seed, it, i, 2);
                    }
                    double len = sqrt(sx * sx + sy * sy + sz * sz);
                    if (len > 0.0) {
                        no[0] = sx / len; /* Eq. 3 with K folded into the renormalisation */
                        no[1] = sy / len;
                        no[2] = sz / len;
                    } else {
                        no[0] = ni[0];
                        no[1] = ni[1];
                        no[2] = ni[2];
                    }
                }
            }
        }
        double* t = cur;
        cur = nxt;
        nxt = t;
    }
    memcpy(Nout, cur, n * sizeof(double));
    free(cur);
    free(nxt);
    return ORC_OK;
}

int orc_bilateral(const double* C, const double* N0, int H, int W, int kernel, double sigma_c,
                  double sigma_s, int iters, double* Nout) {
    return orc_bilateral_jitter(C, N0, H, W, kernel, sigma_c, sigma_s, iters, 0.0, 0, Nout);
}

/* Unit-length copies of the K dominant plane normals (input to Algorithm 4). */
int orc_normalize_dominant(const float* nd, int K, double* out) {
    if (K < 1) return ORC_EINVAL;
    for (int j = 0; j < K; ++j) {
        double x = nd[3 * j], y = nd[3 * j + 1], z = nd[3 * j + 2];
        double len = sqrt(x * x + y * y + z * z);
        if (!(len > 0.0) || !isfinite(len)) return ORC_EINVAL;
        out[3 * j] = x / len;
        out[3 * j + 1] = y / len;
        out[3 * j + 2] = z / len;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 4: group assignment. 255 = no group. best/second receive the    */
/* largest and second-largest dot (for reporting decisions near a threshold).*/
/* ------------------------------------------------------------------------ */
int orc_classify(const double* N, const uint8_t* mask, int64_t n_tri, const double* nd_unit, int K,
                 double ang_min, uint8_t* G, double* best_out, double* second_out) {
    if (K < 1 || K > 254) return ORC_EINVAL;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (int64_t t = 0; t < n_tri; ++t) {
        uint8_t g = 255;
        double best = NAN, second = NAN;
        if (mask[t]) {
            const double* n = N + 3 * t;
            double max_similarity = -1.0;
            for (int j = 0; j < K; ++j) {
                const double* d = nd_unit + 3 * j;
                double s = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
                if (s > max_similarity) {
                    g = (uint8_t)j;
                    max_similarity = s;
                }
            }
            if (max_similarity < ang_min) g = 255;
            /* Diagnostics only: the two largest dots, whatever their sign. */
            best = -INFINITY;
            second = -INFINITY;
            for (int j = 0; j < K; ++j) {
                const double* d = nd_unit + 3 * j;
                double s = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
                if (s > best) {
                    second = best;
                    best = s;
                } else if (s > second) {
                    second = s;
                }
            }
        }
        G[t] = g;
        if (best_out) best_out[t] = best;
        if (second_out) second_out[t] = second;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Twins of Algorithm 2 in T_FC terms: the (up to) three edge neighbours of a */
/* triangle. First (u,v): second (u,v) [diagonal], second (u,v+1) [right],   */
/* second (u-1,v) [top]. Second (u,v): first (u,v) [diagonal], first (u,v-1) */
/* [left], first (u+1,v) [bottom].                                           */
/* ------------------------------------------------------------------------ */
static int tri_twins(int64_t gid, int Hq, int Wq, int64_t out[3]) {
    int k = (int)(gid & 1);
    int64_t q = gid >> 1;
    int u = (int)(q / Wq), v = (int)(q % Wq);
    int n = 0;
    if (k == 0) {
        out[n++] = gid + 1;
        if (v + 1 < Wq) out[n++] = 2 * ((int64_t)u * Wq + v + 1) + 1;
        if (u - 1 >= 0) out[n++] = 2 * ((int64_t)(u - 1) * Wq + v) + 1;
    } else {
        out[n++] = gid - 1;
        if (v - 1 >= 0) out[n++] = 2 * ((int64_t)u * Wq + v - 1);
        if (u + 1 < Hq) out[n++] = 2 * ((int64_t)(u + 1) * Wq + v);
    }
    return n;
}

int orc_triangle_twins(int64_t gid, int H, int W, int64_t* out3) {
    return tri_twins(gid, H - 1, W - 1, out3);
}

/* Algorithm 5: edge-connected region growing inside each group, breadth-first
 * from every unvisited triangle in GID order. Because seeds are taken in
 * increasing GID order, each component's seed is its smallest GID, which is
 * the label. C and nd_unit are only read when max_offset > 0. */
int orc_label(const uint8_t* G, int H, int W, const double* C, const double* nd_unit, int K,
              double max_offset, int tri_min, int32_t* labels) {
    if (H < 2 || W < 2) return ORC_EINVAL;
    const int Hq = H - 1, Wq = W - 1;
    const int64_t n = 2 * (int64_t)Hq * Wq;
    if (n > INT32_MAX) return ORC_EINVAL;
    if (max_offset > 0.0 && (!C || !nd_unit)) return ORC_EINVAL;
    int64_t* queue = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!queue) return ORC_ENOMEM;
    const int32_t UNVISITED = -2;
    for (int64_t t = 0; t < n; ++t) labels[t] = (G[t] == 255) ? -1 : UNVISITED;
    for (int64_t seed = 0; seed < n; ++seed) {
        if (labels[seed] != UNVISITED) continue;
        const uint8_t g = G[seed];
        int64_t head = 0, tail = 0;
        queue[tail++] = seed;
        labels[seed] = (int32_t)seed;
        while (head < tail) {
            int64_t t = queue[head++];
            int64_t nb[3];
            int m = tri_twins(t, Hq, Wq, nb);
            for (int a = 0; a < m; ++a) {
                int64_t j = nb[a];
                if (labels[j] != UNVISITED || G[j] != g) continue;
                if (max_offset > 0.0 && g < K) {
                    const double* d = nd_unit + 3 * g;
                    const double* ct = C + 3 * t;
                    const double* cj = C + 3 * j;
                    double off = d[0] * (ct[0] - cj[0]) + d[1] * (ct[1] - cj[1]) +
                                 d[2] * (ct[2] - cj[2]);
                    if (fabs(off) > max_offset) continue;
                }
                labels[j] = (int32_t)seed;
                queue[tail++] = j;
            }
        }
        /* Algorithm 5 keeps a segment only when |T^g_i| > tri_min. */
        if (tri_min > 0 && tail <= (int64_t)tri_min) {
            for (int64_t a = 0; a < tail; ++a) labels[queue[a]] = -1;
        }
    }
    free(queue);
    return ORC_OK;
}

/* Algorithm 5 with its planarity constraint read as seed-relative: seeds in GID order (every
 * group's task visits its triangles in order, and segments of different groups never meet, so
 * one pass over all groups gives the same result); ExtractPlanarSegment takes the seed and every
 * triangle reachable from it through twin half-edges over triangles of the seed's group that are
 * in no segment yet and whose centroid lies within ptp_max of the plane through the seed's
 * centroid with the group's dominant normal. The triangles of a segment of at most tri_min
 * triangles are dropped (label -1) but stay consumed. Label = the seed's GID, the smallest GID of
 * its segment (every smaller GID of the group was consumed before the seed was reached).
 * margin_out (may be NULL) receives the smallest |offset - ptp_max| over every test made. */
int orc_label_seeded(const uint8_t* G, int H, int W, const double* C, const double* nd_unit, int K, double ptp_max,
                     int tri_min, int32_t* labels, double* margin_out) {
    if (H < 2 || W < 2 || !C || !nd_unit) return ORC_EINVAL;
    const int Hq = H - 1, Wq = W - 1;
    const int64_t n = 2 * (int64_t)Hq * Wq;
    if (n > INT32_MAX) return ORC_EINVAL;
    int64_t* queue = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!queue) return ORC_ENOMEM;
    const int32_t UNVISITED = -2;
    double margin = INFINITY;
    for (int64_t t = 0; t < n; ++t) labels[t] = (G[t] == 255) ? -1 : UNVISITED;
    for (int64_t seed = 0; seed < n; ++seed) {
        if (labels[seed] != UNVISITED) continue;
        const uint8_t g = G[seed];
        const double* d = nd_unit + 3 * (g < K ? g : 0);
        const double* cs = C + 3 * seed;
        int64_t head = 0, tail = 0;
        queue[tail++] = seed;
        labels[seed] = (int32_t)seed;
        while (head < tail) {
            const int64_t t = queue[head++];
            int64_t nb[3];
            const int m = tri_twins(t, Hq, Wq, nb);
            for (int a = 0; a < m; ++a) {
                const int64_t j = nb[a];
                if (labels[j] != UNVISITED || G[j] != g) continue;
                const double* cj = C + 3 * j;
                const double off = fabs(d[0] * (cj[0] - cs[0]) + d[1] * (cj[1] - cs[1]) + d[2] * (cj[2] - cs[2]));
                if (fabs(off - ptp_max) < margin) margin = fabs(off - ptp_max);
                if (off > ptp_max) continue;
                labels[j] = (int32_t)seed;
                queue[tail++] = j;
            }
        }
        if (tri_min > 0 && tail <= (int64_t)tri_min)
            for (int64_t a = 0; a < tail; ++a) labels[queue[a]] = -1;
    }
    if (margin_out) *margin_out = margin;
    free(queue);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: explicit triangle set T (three point indices each, in the    */
/* listed order) and the map T_map from GID to the index in T (-1 if absent).*/
/* Returns the number of triangles.                                          */
/* ------------------------------------------------------------------------ */
int64_t orc_extract_triangles(const double* P_raw, int H, int W, int32_t* T, int32_t* Tmap) {
    if (H < 2 || W < 2) return ORC_EINVAL;
    const int Hq = H - 1, Wq = W - 1;
    int64_t ntri = 0;
    for (int u = 0; u < Hq; ++u) {
        for (int v = 0; v < Wq; ++v) {
            for (int k = 0; k < 2; ++k) {
                int64_t gid = 2 * ((int64_t)u * Wq + v) + k;
                int64_t idx[3];
                tri_vertex_index(u, v, k, W, idx);
                if (isnan(P_raw[3 * idx[0]]) || isnan(P_raw[3 * idx[1]]) ||
                    isnan(P_raw[3 * idx[2]])) {
                    Tmap[gid] = -1;
                    continue;
                }
                T[3 * ntri] = (int32_t)idx[0];
                T[3 * ntri + 1] = (int32_t)idx[1];
                T[3 * ntri + 2] = (int32_t)idx[2];
                Tmap[gid] = (int32_t)ntri;
                ++ntri;
            }
        }
    }
    return ntri;
}

/* Algorithm 2: explicit twin array HE over T (half-edge h belongs to
 * triangle h / 3; -1 = border). Right/Top/Bottom/Left are the neighbouring
 * quads' triangles named in the twin rules above. */
int orc_extract_halfedges(const int32_t* Tmap, int H, int W, int64_t ntri, int32_t* HE) {
    if (H < 2 || W < 2) return ORC_EINVAL;
    const int Hq = H - 1, Wq = W - 1;
    for (int64_t h = 0; h < 3 * ntri; ++h) HE[h] = -1;
    for (int u = 0; u < Hq; ++u) {
        for (int v = 0; v < Wq; ++v) {
            int32_t first = Tmap[2 * ((int64_t)u * Wq + v)];
            int32_t second = Tmap[2 * ((int64_t)u * Wq + v) + 1];
            if (first != -1) {
                int32_t right = (v + 1 < Wq) ? Tmap[2 * ((int64_t)u * Wq + v + 1) + 1] : -1;
                int32_t top = (u - 1 >= 0) ? Tmap[2 * ((int64_t)(u - 1) * Wq + v) + 1] : -1;
                if (right != -1) HE[3 * (int64_t)first] = 3 * right;
                if (top != -1) HE[3 * (int64_t)first + 1] = 3 * top + 1;
                if (second != -1) HE[3 * (int64_t)first + 2] = 3 * second + 2;
            }
            if (second != -1) {
                int32_t left = (v - 1 >= 0) ? Tmap[2 * ((int64_t)u * Wq + v - 1)] : -1;
                int32_t bottom = (u + 1 < Hq) ? Tmap[2 * ((int64_t)(u + 1) * Wq + v)] : -1;
                if (left != -1) HE[3 * (int64_t)second] = 3 * left;
                if (bottom != -1) HE[3 * (int64_t)second + 1] = 3 * bottom + 1;
                if (first != -1) HE[3 * (int64_t)second + 2] = 3 * first + 2;
            }
        }
    }
    return ORC_OK;
}

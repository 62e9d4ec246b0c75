// pl3d_fastga.cu -- the Fast Gaussian Accumulator (Section 6) on the device: the histogram of
// triangle normals over the cells of a refined icosahedron, and peak detection on the host.
//
// Cells (Section 6.1.1). Level 0 is the icosahedron with the 12 vertices (-1, phi, 0),
// (1, phi, 0), (-1, -phi, 0), (1, -phi, 0), (0, -1, phi), (0, 1, phi), (0, -1, -phi),
// (0, 1, -phi), (phi, 0, -1), (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1) (unit length, this order)
// and the 20 faces formed by the triples of mutually adjacent vertices, in lexicographic order of
// the sorted triple, oriented counter-clockwise from outside. Level l + 1 splits face p = (a, b, c)
// into faces 4p .. 4p + 3 = (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca), the midpoints
// projected onto the sphere. A cell's surface normal is its flat face's unit normal.
//
// Search (Section 6.1.3, Algorithm 3). The paper narrows the search with a space-filling-curve
// id, an interpolated window and a binary search, then compares the cell found with its 12
// neighbours. Here every level-0 face is treated as a rotated copy of face 0 (the rotation takes
// the whole refinement with it): the normal's level-0 face comes from the signs and magnitudes of
// its coordinates, the normal is expressed in that face's copy of face 0's frame, and a grid of
// bins over face 0's gnomonic projection holds, per bin, the cells that can be nearest to some
// direction in it (pruned with a bound that is exact for the bin's whole cone of directions, plus
// a margin for FP32 rounding) -- one cell for most bins, a short list compared by dot product as in
// Algorithm 3 otherwise. The host builds these tables once per level from the refinement, and
// checks them: every rotated cell normal must land on a cell normal with the same child numbers.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "pl3d_ctx.cuh"
#include "sync.cuh"

namespace pl3d {
namespace fastga {

constexpr int kMaxLevel = 5;
constexpr int kNbrs = 12;
constexpr int kBinsPerCell = 16;     // bins per cell width along a side of face 0's triangle
constexpr double kPruneEps = 1e-6;

// Host-built tables of one refinement level (device copies live in the context).
struct Tables {
    int level = -1;
    int cells = 0;
    float face0[60];                  // unit normals of the 20 faces of level 0
    std::vector<float> split_planes;  // per face of levels 0..level-1: its 3 inner edge planes (9 floats)
    std::vector<int> level_offset;    // first face of each level in split_planes
    std::vector<float> normals;       // [cells][3] surface normals of the last level
    std::vector<int32_t> nbrs;        // [cells][12] 1-ring neighbours, ascending, -1 padded
    // The canonical frame: face 0's subtree. A rotation of the icosahedron takes face 0 onto
    // face f vertex for vertex, and with it the whole refinement (midpoints projected onto the
    // sphere commute with rotations), child numbers included. So a normal closest to face f is
    // rotated back into face 0's frame, located among face 0's cells, and mapped out again: the
    // device reads tables of one face instead of twenty. Face 0's frame has the basis n0 (its
    // normal), e1, e2; a direction d near face 0 has gnomonic coordinates (d.e1, d.e2) / (d.n0) on
    // a plane where face 0's triangle is a triangle and great circles are lines. A grid of bins over
    // that triangle keeps, per bin, the cells that can be nearest somewhere in it: a cell beaten by
    // another by more than kPruneEps at all four corner directions of a bin is beaten everywhere
    // inside it (the bin's directions are the conic hull of its corners, and the difference of two
    // dot products is linear in the direction). Most bins keep one cell.
    float basis[180];                 // [20][3][3]: R_f n0, R_f e1, R_f e2 (R_f takes face 0 onto face f)
    float pq[2];                      // the level-0 face normals are (+-r, +-r, +-r), r = 1/sqrt(3), and
                                      // the cyclic shifts of (0, +-pq[0], +-pq[1])
    int face_lut[32];                 // [type][sign bits of x, y, z]: the level-0 face (type 0: the
                                      // (+-r, +-r, +-r) normals; 1, 2, 3: the one whose zero is at x, y, z)
    int grid = 0;                     // bins per side
    float g0[2], gs[2];               // bin of (u, v): ((u - g0[0]) gs[0], (v - g0[1]) gs[1])
    std::vector<int32_t> bins;        // [grid * grid], row v: >= 0 the one cell's canonical-set place;
                                      // else -1 - (16 start + count) into multi
    std::vector<float> multi;         // (d.n0, d.e1, d.e2, canonical-set place as int bits) per candidate
    int nc = 0;                       // cells of face 0 (canonical places 0 .. nc - 1 are these cells)
    int n_set = 0;                    // cells of face 0's subtree and their 1-rings
    bool canonical_ok = false;        // every rotated cell normal landed on a cell normal, child numbers kept
    std::vector<int32_t> gmap;        // [20][n_set]: the global cell that candidate s is in face f's frame
};

struct V3d {
    double x, y, z;
};

V3d sub(V3d a, V3d b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3d crs(V3d a, V3d b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V3d unit(V3d a) {
    const double l = sqrt(a.x * a.x + a.y * a.y + a.z * a.z);
    return {a.x / l, a.y / l, a.z / l};
}
double det3(V3d a, V3d b, V3d c) { return a.x * (b.y * c.z - b.z * c.y) - a.y * (b.x * c.z - b.z * c.x) + a.z * (b.x * c.y - b.y * c.x); }

// The cell of the finished tables nearest to direction d, located as the device does (level-0
// face, descent, 1-ring), in double precision; brute force if that is not within 1e-9 of d's own
// direction (only cell normals are located here, and each is its own cell's exactly).
int host_locate(const Tables& t, V3d d) {
    auto dot_at = [&](const float* p) { return d.x * p[0] + d.y * p[1] + d.z * p[2]; };
    int f = 0;
    double best = dot_at(t.face0);
    for (int k = 1; k < 20; ++k)
        if (dot_at(t.face0 + 3 * k) > best) best = dot_at(t.face0 + 3 * k), f = k;
    for (int l = 0; l < t.level; ++l) {
        const float* p = t.split_planes.data() + 9 * ((size_t)t.level_offset[l] + f);
        int c = 3;
        double m = 0.0;
        for (int j = 0; j < 3; ++j)
            if (dot_at(p + 3 * j) > m) m = dot_at(p + 3 * j), c = j;
        f = 4 * f + c;
    }
    int cell = f;
    best = dot_at(t.normals.data() + 3 * (size_t)f);
    for (int k = 0; k < kNbrs; ++k) {
        const int j = t.nbrs[(size_t)f * kNbrs + k];
        if (j >= 0 && dot_at(t.normals.data() + 3 * (size_t)j) > best) best = dot_at(t.normals.data() + 3 * (size_t)j), cell = j;
    }
    if (best > 1.0 - 1e-9) return cell;
    for (int j = 0; j < t.cells; ++j)
        if (dot_at(t.normals.data() + 3 * (size_t)j) > best) best = dot_at(t.normals.data() + 3 * (size_t)j), cell = j;
    return cell;
}

// The canonical-frame tables of t (see Tables). V: the vertices (level-0 ones first), F0: the
// level-0 faces.
void build_canonical(Tables& t, const std::vector<V3d>& V, const std::vector<std::array<int, 3>>& F0) {
    t.canonical_ok = true;
    // the level-0 face normals by type: every one must be (+-r, +-r, +-r) or a cyclic shift of
    // (0, +-p, +-q) with one p, q
    const double r = 1.0 / sqrt(3.0);
    double p = -1.0, q = -1.0;
    for (int f = 0; f < 20 && p < 0.0; ++f)
        if (fabs(t.face0[3 * f]) < 1e-6) p = fabs(t.face0[3 * f + 1]), q = fabs(t.face0[3 * f + 2]);
    t.pq[0] = (float)p;
    t.pq[1] = (float)q;
    for (int k = 0; k < 32; ++k) t.face_lut[k] = -1;
    for (int f = 0; f < 20; ++f) {
        const double n[3] = {t.face0[3 * f], t.face0[3 * f + 1], t.face0[3 * f + 2]};
        int type = -1;
        if (fabs(fabs(n[0]) - r) < 1e-6 && fabs(fabs(n[1]) - r) < 1e-6 && fabs(fabs(n[2]) - r) < 1e-6) type = 0;
        for (int z = 0; z < 3; ++z)   // zero at z; then p at z + 1, q at z + 2 (cyclically)
            if (fabs(n[z]) < 1e-6 && fabs(fabs(n[(z + 1) % 3]) - p) < 1e-6 && fabs(fabs(n[(z + 2) % 3]) - q) < 1e-6)
                type = 1 + z;
        if (type < 0) {
            t.canonical_ok = false;
            continue;
        }
        for (int sb = 0; sb < 8; ++sb) {   // every sign pattern of x, y, z the face's nonzero signs fit
            bool fits = true;
            for (int k = 0; k < 3; ++k)
                if (fabs(n[k]) > 1e-6 && ((n[k] < 0) != (((sb >> k) & 1) != 0))) fits = false;
            if (fits) t.face_lut[8 * type + sb] = f;
        }
    }
    for (int k = 0; k < 32; ++k)
        if (t.face_lut[k] < 0) t.canonical_ok = false;
    // R_f = M_f M_0^-1, M the matrix with a face's vertices as columns
    auto mat = [&](int f, double m[3][3]) {
        for (int c = 0; c < 3; ++c) {
            const V3d& v = V[F0[f][c]];
            m[0][c] = v.x, m[1][c] = v.y, m[2][c] = v.z;
        }
    };
    double m0[3][3], inv[3][3];
    mat(0, m0);
    const double det = m0[0][0] * (m0[1][1] * m0[2][2] - m0[1][2] * m0[2][1]) -
                       m0[0][1] * (m0[1][0] * m0[2][2] - m0[1][2] * m0[2][0]) +
                       m0[0][2] * (m0[1][0] * m0[2][1] - m0[1][1] * m0[2][0]);
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) {
            // inverse = adjugate / det, the adjugate's (i, c) entry the cofactor of (c, i)
            const int r0 = (c + 1) % 3, r1 = (c + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
            inv[i][c] = (m0[r0][c0] * m0[r1][c1] - m0[r0][c1] * m0[r1][c0]) / det;
        }
    std::vector<std::array<double, 9>> R(20);
    for (int f = 0; f < 20; ++f) {
        double m[3][3];
        mat(f, m);
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) {
                double v = 0.0;
                for (int k = 0; k < 3; ++k) v += m[i][k] * inv[k][c];
                R[f][3 * i + c] = v;
            }
    }
    auto rot = [&](int f, V3d w) {
        const double* r = R[f].data();
        return V3d{r[0] * w.x + r[1] * w.y + r[2] * w.z, r[3] * w.x + r[4] * w.y + r[5] * w.z,
                   r[6] * w.x + r[7] * w.y + r[8] * w.z};
    };
    auto dot = [](V3d a, V3d b) { return a.x * b.x + a.y * b.y + a.z * b.z; };
    // face 0's basis; each face's copy of it
    const V3d a0 = V[F0[0][0]], b0 = V[F0[0][1]], c0 = V[F0[0][2]];
    const V3d n0 = unit(crs(sub(b0, a0), sub(c0, a0)));
    const V3d e1 = unit(sub(a0, {n0.x * dot(a0, n0), n0.y * dot(a0, n0), n0.z * dot(a0, n0)}));
    const V3d e2 = crs(n0, e1);
    for (int f = 0; f < 20; ++f) {
        const V3d w[3] = {rot(f, n0), rot(f, e1), rot(f, e2)};
        for (int k = 0; k < 3; ++k) {
            t.basis[9 * f + 3 * k] = (float)w[k].x;
            t.basis[9 * f + 3 * k + 1] = (float)w[k].y;
            t.basis[9 * f + 3 * k + 2] = (float)w[k].z;
        }
    }
    // the canonical set: face 0's cells (ids 0 .. nc - 1: face 0's descendants at any level are
    // the first ids of that level) and their 1-rings
    const int nc = 1 << (2 * t.level);
    t.nc = nc;
    std::vector<int> place(t.cells, -1), set;
    auto add = [&](int j) {
        if (j >= 0 && place[j] < 0) place[j] = 0, set.push_back(j);
    };
    for (int c = 0; c < nc; ++c) {
        add(c);
        for (int k = 0; k < kNbrs; ++k) add(t.nbrs[(size_t)c * kNbrs + k]);
    }
    std::sort(set.begin(), set.end());
    for (size_t i = 0; i < set.size(); ++i) place[set[i]] = (int)i;
    t.n_set = (int)set.size();
    for (int c = 0; c < nc; ++c)
        if (place[c] != c) t.canonical_ok = false;
    auto nrm = [&](int j) { return V3d{t.normals[3 * (size_t)j], t.normals[3 * (size_t)j + 1], t.normals[3 * (size_t)j + 2]}; };
    // the largest angle from a cell normal to its cell's corners: a direction is at most this far
    // from the normal of the cell containing it, so its nearest cell normal is too, and a cell can
    // be nearest only within this angle of its normal
    std::vector<std::array<V3d, 3>> lev = {{a0, b0, c0}};
    for (int d = 0; d < t.level; ++d) {
        std::vector<std::array<V3d, 3>> next;
        for (const auto& f : lev) {
            const V3d a = f[0], b = f[1], c = f[2];
            const V3d ab = unit({a.x + b.x, a.y + b.y, a.z + b.z}), bc = unit({b.x + c.x, b.y + c.y, b.z + c.z}),
                      ca = unit({c.x + a.x, c.y + a.y, c.z + a.z});
            next.push_back({a, ab, ca});
            next.push_back({ab, b, bc});
            next.push_back({ca, bc, c});
            next.push_back({ab, bc, ca});
        }
        lev.swap(next);
    }
    double cos_rmax = 1.0;
    for (int c = 0; c < nc; ++c)
        for (const V3d& v : lev[c]) cos_rmax = std::min(cos_rmax, dot(nrm(c), v));
    const double rmax = acos(std::min(1.0, cos_rmax));
    // the bin grid over face 0's triangle in gnomonic coordinates, 2% wider than its bounding box
    auto gno = [&](V3d d) { return std::array<double, 2>{dot(d, e1) / dot(d, n0), dot(d, e2) / dot(d, n0)}; };
    double lo[2] = {1e30, 1e30}, hi[2] = {-1e30, -1e30};
    for (const V3d& v : {a0, b0, c0}) {
        const auto g = gno(v);
        for (int k = 0; k < 2; ++k) lo[k] = std::min(lo[k], g[k]), hi[k] = std::max(hi[k], g[k]);
    }
    const int G = kBinsPerCell << t.level;
    t.grid = G;
    double step[2];
    for (int k = 0; k < 2; ++k) {
        const double m = 0.01 * (hi[k] - lo[k]);
        lo[k] -= m;
        hi[k] += m;
        step[k] = (hi[k] - lo[k]) / G;
        t.g0[k] = (float)lo[k];
        t.gs[k] = (float)(1.0 / step[k]);
    }
    auto dir = [&](double u, double v) { return unit({n0.x + u * e1.x + v * e2.x, n0.y + u * e1.y + v * e2.y,
                                                      n0.z + u * e1.z + v * e2.z}); };
    std::vector<V3d> setn(set.size());
    for (size_t i = 0; i < set.size(); ++i) setn[i] = nrm(set[i]);
    t.bins.assign((size_t)G * G, 0);
    std::vector<int> cand;
    for (int by = 0; by < G; ++by)
        for (int bx = 0; bx < G; ++bx) {
            const double u0 = lo[0] + bx * step[0], v0 = lo[1] + by * step[1];
            const V3d corner[4] = {dir(u0, v0), dir(u0 + step[0], v0), dir(u0, v0 + step[1]),
                                   dir(u0 + step[0], v0 + step[1])};
            const V3d mid = dir(u0 + 0.5 * step[0], v0 + 0.5 * step[1]);
            double cos_r = 1.0;
            for (const V3d& q : corner) cos_r = std::min(cos_r, dot(mid, q));
            const double reach = cos(std::min(M_PI, acos(std::min(1.0, cos_r)) + rmax) + 1e-9);
            cand.clear();
            for (size_t i = 0; i < set.size(); ++i)
                if (dot(setn[i], mid) >= reach) cand.push_back((int)i);
            std::vector<int> keep;
            for (int jv : cand) {
                bool beaten = false;
                for (size_t k = 0; k < cand.size() && !beaten; ++k) {
                    if (cand[k] == jv) continue;
                    const V3d dd = sub(setn[cand[k]], setn[jv]);
                    beaten = true;
                    for (const V3d& q : corner)
                        if (dot(dd, q) <= kPruneEps) beaten = false;
                }
                if (!beaten) keep.push_back(jv);
            }
            int32_t& e = t.bins[(size_t)by * G + bx];
            if (keep.size() == 1) {
                e = keep[0];
                continue;
            }
            if (keep.empty() || keep.size() > 15) {   // no cell reaches the bin: far outside face 0
                if (keep.empty()) keep.push_back(0);
                else keep.resize(15), t.canonical_ok = false;
            }
            const int start = (int)(t.multi.size() / 4);
            for (int jv : keep) {
                t.multi.push_back((float)dot(setn[jv], n0));
                t.multi.push_back((float)dot(setn[jv], e1));
                t.multi.push_back((float)dot(setn[jv], e2));
                const int32_t pl = jv;
                float w;
                memcpy(&w, &pl, sizeof(w));
                t.multi.push_back(w);
            }
            e = -1 - (16 * start + (int)keep.size());
        }
    t.gmap.resize((size_t)20 * t.n_set);
    for (int f = 0; f < 20; ++f)
        for (int i = 0; i < t.n_set; ++i) {
            const V3d n = nrm(set[i]);
            const double* rr = R[f].data();
            const V3d d = {rr[0] * n.x + rr[1] * n.y + rr[2] * n.z, rr[3] * n.x + rr[4] * n.y + rr[5] * n.z,
                           rr[6] * n.x + rr[7] * n.y + rr[8] * n.z};
            const int g = host_locate(t, d);
            t.gmap[(size_t)f * t.n_set + i] = g;
            // the premise: the image is a cell normal itself, and face 0's cell c is face f's cell c
            const V3d m = nrm(g);
            if (d.x * m.x + d.y * m.y + d.z * m.z < 1.0 - 1e-6) t.canonical_ok = false;
            if (set[i] < nc && g != f * nc + set[i]) t.canonical_ok = false;
        }
}

Tables build(int level) {
    const double phi = (1.0 + sqrt(5.0)) / 2.0;
    const double raw[12][3] = {{-1, phi, 0}, {1, phi, 0}, {-1, -phi, 0}, {1, -phi, 0}, {0, -1, phi}, {0, 1, phi},
                               {0, -1, -phi}, {0, 1, -phi}, {phi, 0, -1}, {phi, 0, 1}, {-phi, 0, -1}, {-phi, 0, 1}};
    std::vector<V3d> V;
    for (auto& r : raw) V.push_back(unit({r[0], r[1], r[2]}));
    auto dist2 = [&](int i, int j) {
        const double dx = raw[i][0] - raw[j][0], dy = raw[i][1] - raw[j][1], dz = raw[i][2] - raw[j][2];
        return dx * dx + dy * dy + dz * dz;
    };
    std::vector<std::array<int, 3>> F;
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j)
            for (int k = j + 1; k < 12; ++k)
                if (fabs(dist2(i, j) - 4) < 1e-9 && fabs(dist2(j, k) - 4) < 1e-9 && fabs(dist2(i, k) - 4) < 1e-9) {
                    const V3d a = {raw[i][0], raw[i][1], raw[i][2]}, b = {raw[j][0], raw[j][1], raw[j][2]},
                              c = {raw[k][0], raw[k][1], raw[k][2]};
                    if (det3(a, b, c) > 0) F.push_back({i, j, k});
                    else F.push_back({i, k, j});
                }
    const std::vector<std::array<int, 3>> F0 = F;   // level-0 faces, vertices 0..11 of V
    Tables t;
    t.level = level;
    for (int i = 0; i < 20; ++i) {
        const V3d n = unit(crs(sub(V[F[i][1]], V[F[i][0]]), sub(V[F[i][2]], V[F[i][0]])));
        t.face0[3 * i] = (float)n.x;
        t.face0[3 * i + 1] = (float)n.y;
        t.face0[3 * i + 2] = (float)n.z;
    }
    for (int l = 0; l < level; ++l) {
        t.level_offset.push_back((int)(t.split_planes.size() / 9));
        std::map<std::pair<int, int>, int> mid;
        auto midpoint = [&](int a, int b) {
            const std::pair<int, int> key(std::min(a, b), std::max(a, b));
            auto it = mid.find(key);
            if (it != mid.end()) return it->second;
            const V3d p = unit({V[a].x + V[b].x, V[a].y + V[b].y, V[a].z + V[b].z});
            V.push_back(p);
            mid[key] = (int)V.size() - 1;
            return (int)V.size() - 1;
        };
        std::vector<std::array<int, 3>> nf;
        nf.reserve(F.size() * 4);
        for (const auto& f : F) {
            const int a = f[0], b = f[1], c = f[2];
            const int ab = midpoint(a, b), bc = midpoint(b, c), ca = midpoint(c, a);
            // the inner edges cutting off the corner children 0 (at a), 1 (at b), 2 (at c): a normal
            // of the face on the positive side of plane j lies in child j, on no positive side in
            // the middle child 3
            const V3d planes[3] = {unit(crs(V[ab], V[ca])), unit(crs(V[bc], V[ab])), unit(crs(V[ca], V[bc]))};
            for (const V3d& p : planes) {
                t.split_planes.push_back((float)p.x);
                t.split_planes.push_back((float)p.y);
                t.split_planes.push_back((float)p.z);
            }
            nf.push_back({a, ab, ca});
            nf.push_back({ab, b, bc});
            nf.push_back({ca, bc, c});
            nf.push_back({ab, bc, ca});
        }
        F.swap(nf);
    }
    t.cells = (int)F.size();
    for (const auto& f : F) {
        const V3d n = unit(crs(sub(V[f[1]], V[f[0]]), sub(V[f[2]], V[f[0]])));
        t.normals.push_back((float)n.x);
        t.normals.push_back((float)n.y);
        t.normals.push_back((float)n.z);
    }
    std::vector<std::vector<int>> inc(V.size());
    for (int i = 0; i < t.cells; ++i)
        for (int v : F[i]) inc[v].push_back(i);
    t.nbrs.assign((size_t)t.cells * kNbrs, -1);
    for (int i = 0; i < t.cells; ++i) {
        std::vector<int> nb;
        for (int v : F[i])
            for (int j : inc[v])
                if (j != i) nb.push_back(j);
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        for (size_t k = 0; k < nb.size() && k < (size_t)kNbrs; ++k) t.nbrs[(size_t)i * kNbrs + k] = nb[k];
    }
    build_canonical(t, V, F0);
    return t;
}

const Tables& tables(int level) {
    static std::mutex mu;
    static Tables cache[kMaxLevel + 1];
    std::lock_guard<std::mutex> lock(mu);
    if (cache[level].level != level) cache[level] = build(level);
    return cache[level];
}

struct GaArgs {
    const float* normals;     // [n][3]
    const uint8_t* mask;      // [n] or nullptr
    long long n;
    long long n_samples;      // ceil(n / stride)
    long long n_iter;         // rounds of kGaBatch samples per thread (the same for every thread)
    int stride;
    int cells;
    int grid;                 // Tables::grid
    int nc;                   // Tables::nc
    int n_set;                // Tables::n_set
    float g0[2], gs[2];       // Tables::g0, gs
    float pq[2];              // Tables::pq
    int face_lut[32];         // Tables::face_lut
    float basis[180];         // Tables::basis (parameter space: one face per warp, mostly)
    const int* bins;          // Tables::bins
    const float4* multi;      // Tables::multi
    const int* gmap;          // [20][n_set]
    int* counts;              // [cells], cleared by the kernel
    int* out_cell;            // [n] or nullptr
    unsigned* barrier;        // the context's grid barrier
    int* error;               // the context's device error word
};

// The cell of unit normal (x, y, z).
//  1. The level-0 face f0 whose normal is closest (for the regular icosahedron each face's
//     spherical triangle is exactly the set of directions closest to its normal): the best of the
//     four normal types against |x|, |y|, |z|, the signs of x, y, z picking the face of that type.
//  2. The normal's coordinates (t, u, v) in face f0's copy of face 0's basis, and its bin at
//     the gnomonic point (u / t, v / t) (t > 0.79 inside a level-0 face).
//  3. The bin's cell, or Algorithm 3's local search -- the closest surface normal -- over the few
//     cells the bin keeps.
//  4. That cell in face f0's frame: face 0's cell c is face f0's cell f0 4^level + c, a cell of
//     the 1-ring outside face 0 is looked up.
__device__ __forceinline__ int ga_cell(const GaArgs& a, float x, float y, float z) {
    const float ax = fabsf(x), ay = fabsf(y), az = fabsf(z);
    const float p = a.pq[0], q = a.pq[1];
    float best = (ax + ay + az) * 0.57735026919f;
    int type = 0;
    const float t1 = ay * p + az * q, t2 = az * p + ax * q, t3 = ax * p + ay * q;
    if (t1 > best) best = t1, type = 1;
    if (t2 > best) best = t2, type = 2;
    if (t3 > best) best = t3, type = 3;
    const int signs = (x < 0.f ? 1 : 0) | (y < 0.f ? 2 : 0) | (z < 0.f ? 4 : 0);
    const int f0 = a.face_lut[8 * type + signs];
    const float* B = a.basis + 9 * f0;
    const float t = B[0] * x + B[1] * y + B[2] * z;
    const float u = B[3] * x + B[4] * y + B[5] * z;
    const float v = B[6] * x + B[7] * y + B[8] * z;
    const float it = __frcp_rn(t);
    const int bx = min(max((int)((u * it - a.g0[0]) * a.gs[0]), 0), a.grid - 1);
    const int by = min(max((int)((v * it - a.g0[1]) * a.gs[1]), 0), a.grid - 1);
    int place = __ldg(a.bins + by * a.grid + bx);
    if (place < 0) {
        const int code = -1 - place;
        const float4* m = a.multi + (code >> 4);
        float4 k = __ldg(m);
        float bd = t * k.x + u * k.y + v * k.z;
        place = __float_as_int(k.w);
        for (int o = 1; o < (code & 15); ++o) {
            k = __ldg(m + o);
            const float dd = t * k.x + u * k.y + v * k.z;
            if (dd > bd) {
                bd = dd;
                place = __float_as_int(k.w);
            }
        }
    }
    return place < a.nc ? f0 * a.nc + place : __ldg(a.gmap + f0 * a.n_set + place);
}

constexpr int kGaThreads = 512;
constexpr int kGaBatch = 2;   // normals a thread loads before it locates them

// One cooperative launch. Every CTA clears its share of the output histogram and loads kGaBatch
// normals per thread before it locates them, counting them in a private histogram; after one grid
// barrier (every share cleared) it adds its histogram to the output.
__global__ void __launch_bounds__(kGaThreads, 2) fastga_kernel(const __grid_constant__ GaArgs a) {
    extern __shared__ int hist[];   // [cells]
    for (int i = threadIdx.x; i < a.cells; i += blockDim.x) hist[i] = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.cells;
         i += (long long)gridDim.x * blockDim.x)
        a.counts[i] = 0;
    __syncthreads();
    const long long n_samples = a.n_samples;
    const long long T = (long long)gridDim.x * blockDim.x;
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    for (long long it = 0; it < a.n_iter; ++it) {
        float x[kGaBatch], y[kGaBatch], z[kGaBatch];
        bool use[kGaBatch], in_range[kGaBatch];
        long long idx[kGaBatch];
#pragma unroll
        for (int k = 0; k < kGaBatch; ++k) {
            const long long s = g + (kGaBatch * it + k) * T;
            in_range[k] = s < n_samples;
            idx[k] = in_range[k] ? s * a.stride : 0;
            x[k] = y[k] = z[k] = NAN;
            if (in_range[k]) {
                x[k] = __ldg(a.normals + 3 * idx[k]);
                y[k] = __ldg(a.normals + 3 * idx[k] + 1);
                z[k] = __ldg(a.normals + 3 * idx[k] + 2);
            }
            use[k] = in_range[k] && (!a.mask || __ldg(a.mask + idx[k]) != 0);
        }
#pragma unroll
        for (int k = 0; k < kGaBatch; ++k) {
            const bool ok = use[k] && isfinite(x[k]) && isfinite(y[k]) && isfinite(z[k]);
            const int cell = ok ? ga_cell(a, x[k], y[k], z[k]) : -1;
            // the warp's first counted cell in one shared-memory atomic, the lanes of other cells
            // one each (neighbouring triangles mostly share a cell)
            const unsigned counted = __ballot_sync(0xffffffffu, cell >= 0);
            if (counted) {
                const int lead = __shfl_sync(0xffffffffu, cell, __ffs(counted) - 1);
                const unsigned same = __ballot_sync(0xffffffffu, cell == lead);
                if (lane == __ffs(counted) - 1) atomicAdd(hist + lead, __popc(same));
                else if (cell >= 0 && cell != lead) atomicAdd(hist + cell, 1);
            }
            if (a.out_cell && in_range[k]) a.out_cell[idx[k]] = cell;
        }
    }
    grid_barrier(a.barrier, a.error);   // every CTA's share of the output cleared (and this CTA's hist final)
    for (int i = threadIdx.x; i < a.cells; i += blockDim.x)
        if (hist[i]) atomicAdd(a.counts + i, hist[i]);
}

}  // namespace fastga
}  // namespace pl3d

using namespace pl3d;
using namespace pl3d::ctxutil;

extern "C" {

int pl3d_fastga_cells(int level, float* out_normals, int32_t* out_neighbors) {
    if (level < 0 || level > fastga::kMaxLevel) return PL3D_ERR_INVALID_ARG;
    const fastga::Tables& t = fastga::tables(level);
    if (!t.canonical_ok) return PL3D_ERR_UNSUPPORTED;   // the tables failed their own check
    if (out_normals) memcpy(out_normals, t.normals.data(), t.normals.size() * sizeof(float));
    if (out_neighbors) memcpy(out_neighbors, t.nbrs.data(), t.nbrs.size() * sizeof(int32_t));
    return t.cells;
}

int pl3d_fastga(pl3d_ctx* ctx, const float* normals, const uint8_t* mask, int64_t n, int level, int stride,
                int32_t* out_counts, int32_t* out_cells, void* stream) {
    if (!ctx || !normals || !out_counts || n < 0 || level < 0 || level > fastga::kMaxLevel || stride < 1)
        return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const fastga::Tables& t = fastga::tables(level);
    if (!t.canonical_ok) return PL3D_ERR_UNSUPPORTED;   // the tables failed their own check
    // device copies of the level's canonical tables, kept by the context
    if (ctx->ga_level != level) {
        if (ctx->ga_tables && cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
        cudaFree(ctx->ga_tables);
        ctx->ga_tables = nullptr;
        ctx->ga_level = -1;
        const void* src[3] = {t.bins.data(), t.multi.data(), t.gmap.data()};
        const size_t bytes[3] = {t.bins.size() * 4, t.multi.size() * 4, t.gmap.size() * 4};
        size_t off[3], total = 0;
        for (int k = 0; k < 3; ++k) {
            off[k] = total;
            total += (bytes[k] + 255) / 256 * 256;
        }
        if (cudaMalloc((void**)&ctx->ga_tables, total) != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_OUT_OF_MEMORY;
        }
        for (int k = 0; k < 3; ++k)
            if (bytes[k] && cudaMemcpy(ctx->ga_tables + off[k], src[k], bytes[k], cudaMemcpyHostToDevice) != cudaSuccess)
                return PL3D_ERR_CUDA;
        ctx->ga_level = level;
        for (int k = 0; k < 3; ++k) ctx->ga_off[k] = off[k];
    }
    // triangles the stride skips are never visited: they read -1 (every byte 0xff)
    if (out_cells && stride > 1 && cudaMemsetAsync(out_cells, 0xff, (size_t)n * sizeof(int32_t), s) != cudaSuccess)
        return PL3D_ERR_CUDA;
    if (n == 0)   // no launch: the histogram is all zeros
        return cudaMemsetAsync(out_counts, 0, (size_t)t.cells * sizeof(int32_t), s) == cudaSuccess ? PL3D_OK
                                                                                                  : PL3D_ERR_CUDA;
    fastga::GaArgs a;
    a.normals = normals;
    a.mask = mask;
    a.n = n;
    a.stride = stride;
    a.cells = t.cells;
    a.grid = t.grid;
    a.nc = t.nc;
    a.n_samples = (n + stride - 1) / stride;
    a.n_set = t.n_set;
    memcpy(a.g0, t.g0, sizeof(a.g0));
    memcpy(a.gs, t.gs, sizeof(a.gs));
    memcpy(a.pq, t.pq, sizeof(a.pq));
    memcpy(a.face_lut, t.face_lut, sizeof(a.face_lut));
    memcpy(a.basis, t.basis, sizeof(a.basis));
    a.bins = reinterpret_cast<const int*>(ctx->ga_tables + ctx->ga_off[0]);
    a.multi = reinterpret_cast<const float4*>(ctx->ga_tables + ctx->ga_off[1]);
    a.gmap = reinterpret_cast<const int*>(ctx->ga_tables + ctx->ga_off[2]);
    a.counts = out_counts;
    a.out_cell = out_cells;
    a.barrier = ctx->barrier();
    a.error = ctx->error();
    const size_t smem = (size_t)t.cells * sizeof(int);
    const void* fn = reinterpret_cast<const void*>(&fastga::fastga_kernel);
    // above the default 48 KB (level 5) the kernel needs the opt-in; set once per level, not per call
    if (smem > 48 * 1024 && ctx->ga_smem_optin < smem) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_CUDA;
        }
        ctx->ga_smem_optin = smem;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PL3D_ERR_CUDA;
    // every resident CTA (one per SM at these sizes): the kernel waits at a grid barrier
    const int grid = resident_ctas(fn, smem, dev, fastga::kGaThreads);
    if (grid <= 0) return PL3D_ERR_CUDA;
    const long long per_round = (long long)fastga::kGaBatch * grid * fastga::kGaThreads;
    a.n_iter = (a.n_samples + per_round - 1) / per_round;
    cudaEvent_t e0, e1;
    record_start(ctx, s, &e0, &e1);
    void* args[1] = {&a};
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(fastga::kGaThreads), args, smem, s) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    record_stop(ctx, s, kSlotFastga, e0, e1);
    ctx->launches += 1;
    return PL3D_OK;
}

int pl3d_fastga_peaks(int level, const int32_t* counts, float v_min, float d_peak, int max_peaks, float* out_normals,
                      int64_t* out_weights) {
    if (level < 0 || level > fastga::kMaxLevel || !counts || max_peaks < 0 || (max_peaks > 0 && !out_normals) ||
        !isfinite(v_min) || !isfinite(d_peak))
        return PL3D_ERR_INVALID_ARG;
    const fastga::Tables& t = fastga::tables(level);
    // a peak: count above v_min, not below any 1-ring neighbour (a plateau keeps its lowest index)
    std::vector<int> pk;
    for (int i = 0; i < t.cells; ++i) {
        if (!((float)counts[i] > v_min)) continue;
        bool peak = true;
        for (int k = 0; k < fastga::kNbrs && peak; ++k) {
            const int j = t.nbrs[(size_t)i * fastga::kNbrs + k];
            if (j >= 0 && !(counts[i] > counts[j] || (counts[i] == counts[j] && i < j))) peak = false;
        }
        if (peak) pk.push_back(i);
    }
    // single-linkage clusters of peaks closer than d_peak; each the count-weighted mean normal
    const int m = (int)pk.size();
    std::vector<int> parent(m);
    for (int i = 0; i < m; ++i) parent[i] = i;
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x];
        return x;
    };
    auto nrm = [&](int c, int d) { return (double)t.normals[3 * (size_t)c + d]; };
    for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j) {
            const double dx = nrm(pk[i], 0) - nrm(pk[j], 0), dy = nrm(pk[i], 1) - nrm(pk[j], 1),
                         dz = nrm(pk[i], 2) - nrm(pk[j], 2);
            if (sqrt(dx * dx + dy * dy + dz * dz) < d_peak) {
                const int ri = find(i), rj = find(j);
                if (ri != rj) parent[std::max(ri, rj)] = std::min(ri, rj);
            }
        }
    struct Cluster {
        double x = 0, y = 0, z = 0;
        int64_t w = 0;
        int first = 1 << 30;
    };
    std::map<int, Cluster> cl;
    for (int i = 0; i < m; ++i) {
        Cluster& c = cl[find(i)];
        const double w = counts[pk[i]];
        c.x += w * nrm(pk[i], 0);
        c.y += w * nrm(pk[i], 1);
        c.z += w * nrm(pk[i], 2);
        c.w += counts[pk[i]];
        c.first = std::min(c.first, pk[i]);
    }
    std::vector<Cluster> out;
    for (auto& kv : cl) out.push_back(kv.second);
    std::sort(out.begin(), out.end(), [](const Cluster& a, const Cluster& b) {
        return a.w != b.w ? a.w > b.w : a.first < b.first;
    });
    const int k = std::min((int)out.size(), max_peaks);
    for (int i = 0; i < k; ++i) {
        const double l = sqrt(out[i].x * out[i].x + out[i].y * out[i].y + out[i].z * out[i].z);
        out_normals[3 * i] = (float)(out[i].x / l);
        out_normals[3 * i + 1] = (float)(out[i].y / l);
        out_normals[3 * i + 2] = (float)(out[i].z / l);
        if (out_weights) out_weights[i] = out[i].w;
    }
    return k;
}

}  // extern "C"

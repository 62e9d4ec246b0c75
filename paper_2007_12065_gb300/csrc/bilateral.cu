// bilateral.cu -- triangle centroids and normals over T_FC (Section 5.2), bilateral normal
// filtering (Eq. 3-6), the triangle mask (Algorithm 1 + the edge predicate of Algorithm 4),
// group assignment (Algorithm 4) and the tile-local part of the planar segments (Algorithm 5),
// fused in one kernel.
//
// Triangles of quad (u, v): first = {p3, p2, p1}, second = {p1, p4, p3} with p1 = (u, v),
// p2 = (u, v+1), p3 = (u+1, v+1), p4 = (u+1, v) (Algorithm 1); normal = (b - a) x (c - a)
// normalised, centroid = (a + b + c) / 3.
//
// Bilateral iteration (Jacobi), for a triangle i with a normal:
//     n_i' = normalize( sum_j W_c(|c_i - c_j|) W_s(|n_i - n_j|) n_j )      (Eq. 3; K cancels)
//     W_c = exp(-|c_i - c_j|^2 / (2 sigma_c^2)),  W_s = exp(-|n_i - n_j|^2 / (2 sigma_s^2))
// over both triangles of every quad in the k x k quad block centred on i's quad, i itself
// included (weight exactly 1), triangles outside the image or without a normal skipped.
// Arithmetic per pair: centroids are stored pre-scaled by sqrt(log2(e) / (2 sigma_c^2)) and,
// for unit normals, |n_i - n_j|^2 = 2 - 2 n_i . n_j, so the product of both exponentials is
// one base-2 exponential of  -|c'_i - c'_j|^2 + a (n_i . n_j - 1),  a = log2(e) / sigma_s^2:
// 3 subtractions, 6 FMAs and one ex2 per pair.
//
// Smoothed points arrive as input position v0 plus displacement d (see df32.cuh). A quad's
// three distinct edge vectors (right p2-p3, diagonal p1-p3, left p4-p1) are first formed in
// FP32 and the normals crossed from them; when an a-priori bound on that FP32 result (from
// the magnitudes of the differences and of the cross product) exceeds 2e-6 rad -- slivers,
// or differences that cancel -- the edges are re-formed as exact float pairs and crossed with
// error-free products instead.
//
// One CTA owns kBilTileH x kBilTileW quads. It stages the smoothed points of its tile plus a
// halo of (fused iterations x radius) quads, builds centroids and normals of every staged
// triangle (and the mask of its own quads), runs the fused iterations in shared memory (the
// valid region shrinks by the radius each iteration; each thread filters two vertically
// adjacent quads, whose windows share most of their loads), and finishes its own quads: mask,
// normal, group, and the connected components of equal group inside the tile. Within a quad
// row the triangles form a chain (second(v) - first(v) across the diagonal, first(v) -
// second(v+1) across the vertical edge), so one warp per row finds the runs of joined
// triangles with ballots and a prefix-max scan (a run's smallest GID is its root); the rows
// are then joined across their horizontal edges with a shared-memory union-find, one union per
// run pair. Each triangle leaves with the GID of its tile-local root; the
// merge kernel in label.cu joins components across tile borders. When the iterations do not
// fit one launch's halo, non-final launches hand their normals to the next through an AoS
// carry buffer.
//
// A triangle without a normal is stored as n = 0, c' = kAbsentCentroid: against any real
// triangle its weight is ex2(-inf) = 0, so it drops out of every sum without a branch.
#include <math.h>

#include "df32.cuh"
#include "pl3d_internal.cuh"
#include "uf.cuh"

namespace pl3d {
namespace {

struct V3 {
    float x, y, z;
};

__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Hardware base-2 exponential (PTX ex2.approx.ftz.f32): subnormal results flush to zero,
// ex2(-inf) = +0.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A staged point: input position and displacement.
struct SP {
    float x, y, z, dx, dy, dz;
};

__device__ __forceinline__ SP load_sp(const float* P, int pplane, int i) {
    return {P[i], P[pplane + i], P[2 * pplane + i], P[3 * pplane + i], P[4 * pplane + i], P[5 * pplane + i]};
}

// Edge b - a as an exact float pair per coordinate.
struct PairEdge {
    F2 x, y, z;
};

__device__ __forceinline__ PairEdge pair_edge(const SP& a, const SP& b) {
    return {pair_diff(a.x, a.dx, b.x, b.dx), pair_diff(a.y, a.dy, b.y, b.dy), pair_diff(a.z, a.dz, b.z, b.dz)};
}

// e1 x e2 from exact pairs, each component rounded once.
__device__ __forceinline__ V3 pair_cross(const PairEdge& e1, const PairEdge& e2) {
    return {pair_sub_round(pair_mul(e1.y, e2.z), pair_mul(e1.z, e2.y)),
            pair_sub_round(pair_mul(e1.z, e2.x), pair_mul(e1.x, e2.z)),
            pair_sub_round(pair_mul(e1.x, e2.y), pair_mul(e1.y, e2.x))};
}

// Edge b - a in FP32 and the size of what was summed to form it (for the error bound).
struct FastEdge {
    V3 e;
    float m;    // sum over coordinates of |v0_b - v0_a| + |d_b - d_a|
    float l1;   // sum over coordinates of |e|
};

__device__ __forceinline__ FastEdge fast_edge(const SP& a, const SP& b) {
    const float ax = b.x - a.x, ay = b.y - a.y, az = b.z - a.z;
    const float dx = b.dx - a.dx, dy = b.dy - a.dy, dz = b.dz - a.dz;
    FastEdge f;
    f.e = {ax + dx, ay + dy, az + dz};
    f.m = (fabsf(ax) + fabsf(dx)) + (fabsf(ay) + fabsf(dy)) + (fabsf(az) + fabsf(dz));
    f.l1 = fabsf(f.e.x) + fabsf(f.e.y) + fabsf(f.e.z);
    return f;
}

__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// The FP32 cross product of two FP32 edges is off by at most about
// 2^-22 sqrt(3) (m1 |e2|_1 + |e1|_1 m2 + |e1|_1 |e2|_1) / |cr|_1 radians; accept it when that
// is below 2e-6 rad (the factor 8 below), otherwise fall back to exact pairs.
__device__ __forceinline__ bool fast_cross_ok(const FastEdge& e1, const FastEdge& e2, V3 cr) {
    const float crl1 = fabsf(cr.x) + fabsf(cr.y) + fabsf(cr.z);
    return e1.m * e2.l1 + e1.l1 * e2.m + e1.l1 * e2.l1 <= 8.f * crl1;
}

__device__ __forceinline__ V3 centroid3(const SP& a, const SP& b, const SP& c) {
    const float k = 1.f / 3.f;
    return {((a.x + b.x + c.x) + (a.dx + b.dx + c.dx)) * k, ((a.y + b.y + c.y) + (a.dy + b.dy + c.dy)) * k,
            ((a.z + b.z + c.z) + (a.dz + b.dz + c.dz)) * k};
}

// Per-quad records in shared memory: 6 floats (triangle 0 xyz, triangle 1 xyz) read and
// written as three float2.
__device__ __forceinline__ void load_quad(const float* A, int q, V3& t0, V3& t1) {
    const float2* a = reinterpret_cast<const float2*>(A) + 3 * q;
    const float2 u = a[0], v = a[1], w = a[2];
    t0 = {u.x, u.y, v.x};
    t1 = {v.y, w.x, w.y};
}

__device__ __forceinline__ void store_quad(float* A, int q, V3 t0, V3 t1) {
    float2* a = reinterpret_cast<float2*>(A) + 3 * q;
    a[0] = make_float2(t0.x, t0.y);
    a[1] = make_float2(t0.z, t1.x);
    a[2] = make_float2(t1.y, t1.z);
}

__device__ __forceinline__ bool has_normal(V3 n) { return n.x != 0.f || n.y != 0.f || n.z != 0.f; }

__device__ __forceinline__ V3 finish_normal(V3 s, V3 own) {
    const float l2 = dot(s, s);
    if (!has_normal(own) || !(l2 > 0.f)) return own;
    const float inv = rsqrtf(l2);
    return {s.x * inv, s.y * inv, s.z * inv};
}

// One pair (i, j): s_i += W n_j with W = ex2(-|c'_i - c'_j|^2 + p_i . n_j - a), p_i = a n_i.
__device__ __forceinline__ void accumulate(V3& s, V3 ci, V3 pi, float a, V3 cj, V3 nj) {
    const float dx = ci.x - cj.x, dy = ci.y - cj.y, dz = ci.z - cj.z;
    float e = fmaf(pi.x, nj.x, fmaf(pi.y, nj.y, fmaf(pi.z, nj.z, -a)));
    e = fmaf(-dx, dx, fmaf(-dy, dy, fmaf(-dz, dz, e)));
    const float w = ex2(e);
    s.x = fmaf(w, nj.x, s.x);
    s.y = fmaf(w, nj.y, s.y);
    s.z = fmaf(w, nj.z, s.z);
}

// State of one quad being filtered.
struct QuadAcc {
    V3 c0, c1;   // scaled centroids
    V3 n0, n1;   // current normals
    V3 p0, p1;   // a * normals
    V3 s0, s1;   // weighted sums
};

__device__ __forceinline__ void quad_begin(QuadAcc& A, const float* Cq, const float* cur, int q, float a) {
    load_quad(Cq, q, A.c0, A.c1);
    load_quad(cur, q, A.n0, A.n1);
    A.p0 = {a * A.n0.x, a * A.n0.y, a * A.n0.z};
    A.p1 = {a * A.n1.x, a * A.n1.y, a * A.n1.z};
    // the triangle itself (weight exactly 1) and its partner in the quad
    A.s0 = A.n0;
    A.s1 = A.n1;
    accumulate(A.s0, A.c0, A.p0, a, A.c1, A.n1);
    accumulate(A.s1, A.c1, A.p1, a, A.c0, A.n0);
}

__device__ __forceinline__ void quad_neighbour(QuadAcc& A, float a, V3 cj0, V3 cj1, V3 nj0, V3 nj1) {
    accumulate(A.s0, A.c0, A.p0, a, cj0, nj0);
    accumulate(A.s0, A.c0, A.p0, a, cj1, nj1);
    accumulate(A.s1, A.c1, A.p1, a, cj0, nj0);
    accumulate(A.s1, A.c1, A.p1, a, cj1, nj1);
}

template <int R, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kBilThreads) bilateral_kernel(BilArgs a) {
    constexpr int TH = kBilTileH, TW = kBilTileW;
    static_assert(TW == 32, "the row-run labeling maps one quad column to one lane");
    static_assert(kBilThreads % 32 == 0, "whole warps");
    extern __shared__ __align__(16) float smem[];
    const int halo = a.iters * R;
    const int RQH = TH + 2 * halo;             // staged quads
    const int RQW = TW + 2 * halo;
    const int PW = RQW + 1;                    // staged points
    const int pplane = (RQH + 1) * PW;
    const int nq = RQH * RQW;
    const int nqs = nq + RQW;                  // plus one spare row: a strip's second quad never reads past it
    float* Cq = smem;                          // [nqs][6] scaled centroids
    float* Na = Cq + 6 * nqs;                  // [nqs][6] normals
    float* Nb = Na + 6 * nqs;                  // [nqs][6] normals; the staged points before the iterations
    float* P = Nb;                             // [6][RQH+1][RQW+1]: v0 x, y, z, d x, y, z
    const int xwords = 6 * nqs > 6 * pplane ? 6 * nqs : 6 * pplane;
    uint8_t* Mk = reinterpret_cast<uint8_t*>(Nb + xwords);      // [TH*TW*2] own masks
    uint8_t* Gs = Mk + 2 * TH * TW;                             // [TH*TW*2] own groups
    const int H = a.H, W = a.W, Hq = H - 1, Wq = W - 1;
    const int qu0 = blockIdx.y * TH - halo;
    const int qv0 = blockIdx.x * TW - halo;
    const float cs = a.c_scale;

    for (int i = threadIdx.x; i < pplane; i += blockDim.x) {
        const int r = i / PW, c = i - r * PW;
        const int gu = qu0 + r, gv = qv0 + c;
        float x = NAN, y = NAN, z = NAN, dx = 0.f, dy = 0.f, dz = 0.f;
        if (gu >= 0 && gu < H && gv >= 0 && gv < W) {
            const size_t p = (size_t)gu * W + gv;
            x = __ldg(a.points + 3 * p);
            y = __ldg(a.points + 3 * p + 1);
            z = __ldg(a.points + 3 * p + 2);
            if (!point_valid(x, y, z)) x = y = z = NAN;
            dx = __ldg(a.dx + p);
            dy = __ldg(a.dy + p);
            dz = __ldg(a.dz + p);
        }
        P[i] = x;
        P[pplane + i] = y;
        P[2 * pplane + i] = z;
        P[3 * pplane + i] = dx;
        P[4 * pplane + i] = dy;
        P[5 * pplane + i] = dz;
    }
    __syncthreads();

    // Centroids and normals of every staged triangle; masks of the CTA's own quads. Results go
    // to Cq and Na only: P (aliased with Nb) stays intact until the barrier below.
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int qr = q / RQW, qc = q - qr * RQW;
        const int gu = qu0 + qr, gv = qv0 + qc;
        const bool exists = gu >= 0 && gu < Hq && gv >= 0 && gv < Wq;
        const int i1 = qr * PW + qc, i2 = i1 + 1, i3 = i1 + PW + 1, i4 = i1 + PW;
        const SP p1 = load_sp(P, pplane, i1), p2 = load_sp(P, pplane, i2);
        const SP p3 = load_sp(P, pplane, i3), p4 = load_sp(P, pplane, i4);
        const bool own = LAST && qr >= halo && qr < halo + TH && qc >= halo && qc < halo + TW;
        const bool v1 = p1.x == p1.x, v2 = p2.x == p2.x, v3 = p3.x == p3.x, v4 = p4.x == p4.x;
        const bool valid0 = exists && v1 && v2 && v3;                            // Algorithm 1
        const bool valid1 = exists && v1 && v3 && v4;
        V3 nn[2] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        if (FIRST) {
            // first = {p3, p2, p1}: (p2 - p3) x (p1 - p3);  second = {p1, p4, p3}: (p4 - p1) x (p3 - p1)
            const FastEdge er = fast_edge(p3, p2), ed = fast_edge(p3, p1), el = fast_edge(p1, p4);
            const FastEdge edn = {{-ed.e.x, -ed.e.y, -ed.e.z}, ed.m, ed.l1};
            V3 cr0 = cross(er.e, ed.e), cr1 = cross(el.e, edn.e);
            const bool exact0 = valid0 && !fast_cross_ok(er, ed, cr0);
            const bool exact1 = valid1 && !fast_cross_ok(el, edn, cr1);
            if (exact0 || exact1) {
                const PairEdge pd = pair_edge(p3, p1);
                if (exact0) cr0 = pair_cross(pair_edge(p3, p2), pd);
                if (exact1) {
                    const PairEdge pdn = {{-pd.x.h, -pd.x.l}, {-pd.y.h, -pd.y.l}, {-pd.z.h, -pd.z.l}};
                    cr1 = pair_cross(pair_edge(p1, p4), pdn);
                }
            }
            const V3 cr[2] = {cr0, cr1};
            const bool vk[2] = {valid0, valid1};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float len2 = dot(cr[k], cr[k]);
                if (vk[k] && len2 > kDegenerateLen2) {
                    const float inv = rsqrtf(len2);
                    nn[k] = {cr[k].x * inv, cr[k].y * inv, cr[k].z * inv};
                }
            }
        } else {
            const bool vk[2] = {valid0, valid1};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!vk[k]) continue;
                const size_t gid = 2 * ((size_t)gu * Wq + gv) + k;
                const float nx = __ldg(a.carry_in + 3 * gid);
                if (nx == nx) nn[k] = {nx, __ldg(a.carry_in + 3 * gid + 1), __ldg(a.carry_in + 3 * gid + 2)};
            }
        }
        V3 cc[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const SP& va = k == 0 ? p3 : p1;
            const SP& vb = k == 0 ? p2 : p4;
            const SP& vc = k == 0 ? p1 : p3;
            cc[k] = {kAbsentCentroid, kAbsentCentroid, kAbsentCentroid};
            if (has_normal(nn[k])) {
                const V3 c0 = centroid3(va, vb, vc);
                cc[k] = {c0.x * cs, c0.y * cs, c0.z * cs};
            }
        }
        if (own) {                                                               // Algorithm 4, l_max
            // edges in FP32: an error of ~1e-7 relative is far inside the 1e-5 m band where
            // FP32 and FP64 may disagree
            const V3 er = fast_edge(p3, p2).e, et = fast_edge(p2, p1).e, ed = fast_edge(p3, p1).e;
            const V3 el = fast_edge(p1, p4).e, eb = fast_edge(p4, p3).e;
            const float d2 = dot(ed, ed);
            const float l0 = fmaxf(d2, fmaxf(dot(er, er), dot(et, et)));
            const float l1 = fmaxf(d2, fmaxf(dot(el, el), dot(eb, eb)));
            const int t = 2 * ((qr - halo) * TW + (qc - halo));
            Mk[t] = (valid0 && l0 <= a.max_edge2) ? 1 : 0;
            Mk[t + 1] = (valid1 && l1 <= a.max_edge2) ? 1 : 0;
        }
        store_quad(Cq, q, cc[0], cc[1]);
        store_quad(Na, q, nn[0], nn[1]);
    }
    __syncthreads();   // the staged points are dead from here on; Nb reuses their space

    // Fused bilateral iterations: each work item is a vertical pair of quads.
    float* cur = Na;
    float* nxt = Nb;
    const float an = a.a_norm;
    for (int it = 1; it <= a.iters; ++it) {
        const int lo = it * R;
        const int ch = RQH - 2 * lo, cw = RQW - 2 * lo;
        const int strips = (ch + 1) >> 1;
        for (int i = threadIdx.x; i < strips * cw; i += blockDim.x) {
            const int sr = i / cw;
            const int qr = lo + 2 * sr, qc = lo + (i - sr * cw);
            const bool two = qr + 1 < RQH - lo;
            const int qA = qr * RQW + qc, qB = qA + RQW;
            // Both quads are always computed (a missing second quad reads the spare row and is
            // not stored), so the unrolled window below has no data-dependent branch.
            QuadAcc A, B;
            quad_begin(A, Cq, cur, qA, an);
            quad_begin(B, Cq, cur, qB, an);
#pragma unroll
            for (int dr = -R; dr <= R + 1; ++dr) {
#pragma unroll
                for (int dc = -R; dc <= R; ++dc) {
                    const bool forA = dr <= R && !(dr == 0 && dc == 0);
                    const bool forB = dr >= 1 - R && !(dr == 1 && dc == 0);
                    const int qj = qA + dr * RQW + dc;
                    V3 cj0, cj1, nj0, nj1;
                    load_quad(Cq, qj, cj0, cj1);
                    load_quad(cur, qj, nj0, nj1);
                    if (forA) quad_neighbour(A, an, cj0, cj1, nj0, nj1);
                    if (forB) quad_neighbour(B, an, cj0, cj1, nj0, nj1);
                }
            }
            store_quad(nxt, qA, finish_normal(A.s0, A.n0), finish_normal(A.s1, A.n1));
            if (two) store_quad(nxt, qB, finish_normal(B.s0, B.n0), finish_normal(B.s1, B.n1));
        }
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }

    // Own quads: hand the normals on, or finish them.
    if (!LAST) {
        for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
            const int r = i / TW, c = i - r * TW;
            const int gu = blockIdx.y * TH + r, gv = blockIdx.x * TW + c;
            if (gu >= Hq || gv >= Wq) continue;
            V3 n[2];
            load_quad(cur, (r + halo) * RQW + (c + halo), n[0], n[1]);
            const size_t gid0 = 2 * ((size_t)gu * Wq + gv);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const bool has = has_normal(n[k]);
                float* o = a.carry_out + 3 * (gid0 + k);
                o[0] = has ? n[k].x : NAN;
                o[1] = has ? n[k].y : NAN;
                o[2] = has ? n[k].z : NAN;
            }
        }
        return;
    }

    int32_t* Lp = reinterpret_cast<int32_t*>(nxt);   // free after the last iteration: [TH*TW*2] parents
    for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
        const int r = i / TW, c = i - r * TW;
        const int gu = blockIdx.y * TH + r, gv = blockIdx.x * TW + c;
        const bool exists = gu < Hq && gv < Wq;
        V3 n[2];
        load_quad(cur, (r + halo) * RQW + (c + halo), n[0], n[1]);
        const size_t gid0 = exists ? 2 * ((size_t)gu * Wq + gv) : 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int t = 2 * i + k;
            const bool kept = Mk[t] != 0;
            const bool has = has_normal(n[k]);
            int g = PL3D_NO_GROUP;
            if (exists && kept && has) {                                         // Algorithm 4, ang_min
                float best = -1.0f;
                for (int j = 0; j < a.nd.K; ++j) {
                    const float s = n[k].x * a.nd.v[3 * j] + n[k].y * a.nd.v[3 * j + 1] + n[k].z * a.nd.v[3 * j + 2];
                    if (s > best) {
                        best = s;
                        g = j;
                    }
                }
                if (best < a.min_dot) g = PL3D_NO_GROUP;
            }
            if (exists) {
                const size_t gid = gid0 + k;
                a.out_mask[gid] = kept ? 1 : 0;
                float* o = a.out_normals + 3 * gid;
                o[0] = has ? n[k].x : NAN;
                o[1] = has ? n[k].y : NAN;
                o[2] = has ? n[k].z : NAN;
                a.out_groups[gid] = (uint8_t)g;
                if (a.sizes) a.sizes[gid] = 0;
            }
            Gs[t] = exists ? (uint8_t)g : (uint8_t)PL3D_NO_GROUP;
        }
    }
    __syncthreads();

    // Connected components inside the tile (twins of Algorithm 2 that stay in the tile).
    // Offset test between a first triangle and a second triangle (scaled centroids).
    const bool offs = a.max_offset_scaled > 0.f;
    const float lim = a.max_offset_scaled;
    auto offset_ok = [&](int g, V3 ci, V3 cj) {
        const float* nd = a.nd.v + 3 * g;
        return !offs || fabsf(nd[0] * (ci.x - cj.x) + nd[1] * (ci.y - cj.y) + nd[2] * (ci.z - cj.z)) <= lim;
    };
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // (1) Runs along each quad row. Chain position 2v is second(v), 2v+1 is first(v).
    for (int r = warp; r < TH; r += kBilThreads / 32) {
        const int tf = 2 * (r * TW + lane), ts = tf + 1;
        const int gf = Gs[tf], gs = Gs[ts];
        V3 cf = {0.f, 0.f, 0.f}, cs2 = cf;
        if (offs) load_quad(Cq, (r + halo) * RQW + (lane + halo), cf, cs2);
        const int gs_next = __shfl_down_sync(kFull, gs, 1);
        const V3 cs_next = {__shfl_down_sync(kFull, cs2.x, 1), __shfl_down_sync(kFull, cs2.y, 1),
                            __shfl_down_sync(kFull, cs2.z, 1)};
        const bool diag = gf != PL3D_NO_GROUP && gs == gf && offset_ok(gf, cf, cs2);
        const bool right = lane < 31 && gf != PL3D_NO_GROUP && gs_next == gf && offset_ok(gf, cf, cs_next);
        const bool right_prev = __shfl_up_sync(kFull, right, 1);
        const bool brk_s = lane == 0 || !right_prev;                 // a run starts at second(v)
        const bool brk_f = !diag;                                    // a run starts at first(v)
        int pm = brk_f ? 2 * lane + 1 : (brk_s ? 2 * lane : -1);      // last run start up to this lane
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, pm, o);
            if (lane >= o) pm = max(pm, v);
        }
        const int before = __shfl_up_sync(kFull, pm, 1);
        const int start_s = brk_s ? 2 * lane : before;
        const int start_f = pm;
        const unsigned brk_f_mask = __ballot_sync(kFull, brk_f);
        // smallest GID of a run starting at chain position p: first(p/2), unless the run is
        // second(p/2) alone
        auto root_of = [&](int p) {
            const int l0 = p >> 1;
            const int t0 = 2 * (r * TW + l0);
            return ((p & 1) || !((brk_f_mask >> l0) & 1u)) ? t0 : t0 + 1;
        };
        Lp[ts] = gs != PL3D_NO_GROUP ? root_of(start_s) : -1;
        Lp[tf] = gf != PL3D_NO_GROUP ? root_of(start_f) : -1;
    }
    __syncthreads();
    // (2) Rows joined across horizontal edges: first(r, v) with second(r-1, v); one union per
    // run pair (a lane skips the pair its left neighbour already joined).
    for (int r = 1 + warp; r < TH; r += kBilThreads / 32) {
        const int tf = 2 * (r * TW + lane), tu = 2 * ((r - 1) * TW + lane) + 1;
        const int gf = Gs[tf];
        bool link = gf != PL3D_NO_GROUP && Gs[tu] == gf;
        if (offs && link) {
            V3 cf, c1, c0u, cu;
            load_quad(Cq, (r + halo) * RQW + (lane + halo), cf, c1);
            load_quad(Cq, (r - 1 + halo) * RQW + (lane + halo), c0u, cu);
            link = offset_ok(gf, cf, cu);
        }
        const int ra = link ? Lp[tf] : -1, rb = link ? Lp[tu] : -1;
        const int pa = __shfl_up_sync(kFull, ra, 1), pb = __shfl_up_sync(kFull, rb, 1);
        const bool dup = lane > 0 && pa == ra && pb == rb;
        if (link && !dup) uf_unite(Lp, ra, rb);
    }
    __syncthreads();

    // Each triangle leaves with the GID of its tile-local root (-1 without a group).
    for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
        const int r = i / TW, c = i - r * TW;
        const int gu = blockIdx.y * TH + r, gv = blockIdx.x * TW + c;
        if (gu >= Hq || gv >= Wq) continue;
        const size_t gid0 = 2 * ((size_t)gu * Wq + gv);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int t = 2 * i + k;
            int lab = -1;
            if (Lp[t] >= 0) {
                const int root = uf_root(Lp, t);
                const int rq = root >> 1, rr = rq / TW, rc = rq - rr * TW;
                lab = (int)(2 * ((size_t)(blockIdx.y * TH + rr) * Wq + (blockIdx.x * TW + rc)) + (root & 1));
            }
            a.out_labels[gid0 + k] = lab;
        }
    }
}

template <int R, bool FIRST, bool LAST>
cudaError_t launch_rfl(const BilArgs& a, cudaStream_t s) {
    dim3 grid(div_up(a.W - 1, kBilTileW), div_up(a.H - 1, kBilTileH));
    bilateral_kernel<R, FIRST, LAST><<<grid, kBilThreads, bilateral_smem_bytes(R, a.iters), s>>>(a);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_r(const BilArgs& a, bool first, bool last, cudaStream_t s) {
    if (first && last) return launch_rfl<R, true, true>(a, s);
    if (first) return launch_rfl<R, true, false>(a, s);
    if (last) return launch_rfl<R, false, true>(a, s);
    return launch_rfl<R, false, false>(a, s);
}

template <int R>
cudaError_t configure_r() {
    const int bytes = (int)bilateral_smem_bytes(R, kBilMaxHalo / R);
    cudaError_t e = cudaFuncSetAttribute(bilateral_kernel<R, true, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bilateral_kernel<R, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bilateral_kernel<R, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bilateral_kernel<R, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    return e;
}

}  // namespace

size_t bilateral_smem_bytes(int radius, int iters) {
    const size_t halo = (size_t)iters * radius;
    const size_t rqh = kBilTileH + 2 * halo, rqw = kBilTileW + 2 * halo;
    const size_t nqs = rqh * rqw + rqw;
    const size_t points = 6 * (rqh + 1) * (rqw + 1);
    const size_t x = points > 6 * nqs ? points : 6 * nqs;
    return (12 * nqs + x) * sizeof(float) + 4 * (size_t)kBilTileH * kBilTileW;
}

void bilateral_scales(float sigma_c, float sigma_s, int iters, float* c_scale, float* a_norm) {
    const double log2e = 1.4426950408889634;
    double cs = 1.0, an = 0.0;
    if (iters > 0) {
        cs = sqrt(log2e / (2.0 * (double)sigma_c * (double)sigma_c));
        an = log2e / ((double)sigma_s * (double)sigma_s);
    }
    // finite and representable: c' = c * cs must not overflow for coordinates up to ~1e18
    *c_scale = (float)fmin(fmax(cs, 1e-18), 1e18);
    *a_norm = (float)fmin(an, 1e30);
}

cudaError_t bilateral_configure() {
    cudaError_t e = configure_r<1>();
    if (e == cudaSuccess) e = configure_r<2>();
    if (e == cudaSuccess) e = configure_r<3>();
    return e;
}

cudaError_t launch_bilateral(const BilArgs& a, int radius, bool first, bool last, cudaStream_t s) {
    switch (radius) {
        case 1: return launch_r<1>(a, first, last, s);
        case 2: return launch_r<2>(a, first, last, s);
        case 3: return launch_r<3>(a, first, last, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pl3d

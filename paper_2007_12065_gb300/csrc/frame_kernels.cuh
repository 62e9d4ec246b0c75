// frame_kernels.cuh -- the whole path for one frame in one persistent, cooperatively launched
// kernel: Laplacian tiles -> grid barrier -> bilateral tiles (normals, filter, mask, groups,
// tile-local segments) -> grid barrier -> segment merge across tile borders -> grid barrier ->
// labels (and the tri_min filter). Each CTA loops over the tiles of a phase; the grid barrier
// (sync.cuh) orders the phases. Included once per (Laplacian radius, bilateral radius).
//
// Bilateral arithmetic (Eq. 3-6): centroids are stored pre-scaled by sqrt(log2(e) / (2 sigma_c^2))
// and, for unit normals, |n_i - n_j|^2 = 2 - 2 n_i . n_j, so W_c W_s for a pair is one base-2
// exponential of -(|c'_i - c'_j|^2 + a - a n_i . n_j), a = log2(e) / sigma_s^2; a triangle is
// filtered against both triangles of a neighbour quad at once with paired FP32 instructions.
//
// Tiles are staged from HBM with TMA: the input points and the displacements are both AoS
// [H][W][3] floats, seen as 2-D tensors of H rows x 3W floats, so one box per array covers a
// tile plus its halo (points outside the image read as NaN, displacements as 0). The box's x
// coordinate is rounded down to a 16-byte boundary; `delta` is the float offset of the tile's
// first point inside a box row. When TMA cannot be used (W not a multiple of 4, a misaligned
// pointer, or a phase split into several launches' worth of iterations), the same box is
// filled with plain loads, so everything after staging is identical.
#pragma once

#include <math.h>

#include "df32.cuh"
#include "f32x2.cuh"
#include "pl3d_internal.cuh"
#include "sync.cuh"
#include "uf.cuh"

namespace pl3d {
namespace frame {

constexpr int T = kTile;   // tile edge: points (Laplacian) or quads (bilateral)

struct V3 {
    float x, y, z;
};

__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// Hardware approximations from the PTX ISA: base-2 exponential (ex2(-inf) = +0, subnormal
// results flush to zero) and reciprocal square root (rsqrt(+inf) = 0), both within 2 ulp.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Floor of x to a multiple of 4 (also for negative x).
__device__ __forceinline__ int floor4(int x) { return x & ~3; }

// ------------------------------------------------------------------------------------ staging

// Fills the box rows x cols (floats) whose top-left element is (x0, y0) of the AoS array
// `src` seen as H rows of 3W floats: TMA when `map` is given, else plain loads. Elements
// outside the array read as `fill`. `bar` completes when the TMA bytes have landed.
__device__ __forceinline__ void stage_box(float* dst, const float* src, const CUtensorMap* map, const BoxGeom& b,
                                          int x0, int y0, int H, int W, float fill, uint64_t* bar, int n_tma_boxes,
                                          bool issue_tma) {
    if (map) {
        if (issue_tma && threadIdx.x == 0) {
            if (n_tma_boxes > 0) mbar_arrive_expect_tx(bar, (unsigned)(n_tma_boxes * b.rows * b.cols * 4));
            tma_load_2d(dst, map, x0, y0, bar);
        }
        return;
    }
    const int row_floats = 3 * W;
    for (int e = threadIdx.x; e < b.rows * b.cols; e += blockDim.x) {
        const int r = e / b.cols, x = e - r * b.cols;
        const int gy = y0 + r, gx = x0 + x;
        float v = fill;
        // L2-coherent loads: displacements were written earlier in this launch by other CTAs,
        // and a non-coherent (read-only) cache line from an earlier pass could be stale
        if (src && gy >= 0 && gy < H && gx >= 0 && gx < row_floats) v = __ldcg(src + (size_t)gy * row_floats + gx);
        dst[e] = v;
    }
}

// ------------------------------------------------------------------------------ Laplacian

// A Jacobi iteration updates strips of kLapStrip vertically adjacent points per thread: the
// strip shares the loads of its (kLapStrip + 2R) x (2R + 1) window, and two strip points closer
// than the radius share one weight (w_ij = w_ji, opposite differences).
constexpr int kLapStrip = 4;

// A point as an iteration sees it: input position (invalid -> kInvalidCoord) and displacement.
struct LapPt {
    float x, y, z, dx, dy, dz;
};

// WITH_D = false: the displacement is zero everywhere (the first iteration of the first pass),
// so it is neither loaded nor summed -- the same values as adding zeros.
template <bool WITH_D>
__device__ __forceinline__ LapPt lap_load(const float* V0, const float* D, int o) {
    LapPt p;
    p.x = V0[o];
    p.y = V0[o + 1];
    p.z = V0[o + 2];
    if (WITH_D) {
        p.dx = D[o];
        p.dy = D[o + 1];
        p.dz = D[o + 2];
    } else {
        p.dx = p.dy = p.dz = 0.f;
    }
    return p;
}

struct LapAcc {
    LapPt c;                     // centre
    float sx, sy, sz, ws;        // weighted sums
};

// The Laplacian arithmetic below is written with explicit rounding intrinsics (no contraction
// left to the compiler), so that every kernel that evaluates Eq. 1-2 -- the fused tile passes and
// the single-iteration pass (lap1.cu) -- gives the same bits for the same point.

// Difference q - p of two smoothed points, input and displacement parts subtracted separately.
template <bool WITH_D>
__device__ __forceinline__ void lap_diff(const LapPt& p, const LapPt& q, float& ex, float& ey, float& ez) {
    if (WITH_D) {
        ex = __fadd_rn(__fsub_rn(q.x, p.x), __fsub_rn(q.dx, p.dx));
        ey = __fadd_rn(__fsub_rn(q.y, p.y), __fsub_rn(q.dy, p.dy));
        ez = __fadd_rn(__fsub_rn(q.z, p.z), __fsub_rn(q.dz, p.dz));
    } else {
        ex = __fsub_rn(q.x, p.x);
        ey = __fsub_rn(q.y, p.y);
        ez = __fsub_rn(q.z, p.z);
    }
}

// Eq. 2: w = 1 / |v_j - v|; a neighbour at distance 0 is skipped. An invalid point holds
// kInvalidCoord: the squared distance overflows to +inf and rsqrt(+inf) = 0. A difference and its
// negation give the same weight (w_ij = w_ji).
__device__ __forceinline__ float lap_weight(float ex, float ey, float ez) {
    const float d2 = fmaf(ez, ez, fmaf(ey, ey, __fmul_rn(ex, ex)));
    return d2 > 0.f ? rsqrt_approx(d2) : 0.f;
}

// s += w e for a neighbour difference e and its weight w (the centre's sums of Eq. 1).
__device__ __forceinline__ void lap_accumulate(float& sx, float& sy, float& sz, float& ws, float w, float ex, float ey,
                                               float ez) {
    sx = fmaf(w, ex, sx);
    sy = fmaf(w, ey, sy);
    sz = fmaf(w, ez, sz);
    ws = __fadd_rn(ws, w);
}

template <bool WITH_D>
__device__ __forceinline__ void lap_add(LapAcc& A, const LapPt& q) {
    float ex, ey, ez;
    lap_diff<WITH_D>(A.c, q, ex, ey, ez);
    lap_accumulate(A.sx, A.sy, A.sz, A.ws, lap_weight(ex, ey, ez), ex, ey, ez);
}

// Eq. 1 on the displacement of a centre point: d' = d + (lambda / W) s, or d unchanged (keep).
__device__ __forceinline__ float lap_scale(bool keep, float lambda, float ws) {
    return keep ? 0.f : __fdividef(lambda, ws);
}

// Top-left element (x0, u0) of a Laplacian tile's box in the AoS array seen as H rows of 3W
// floats, and the offset of the tile's first point inside its box row. Tiles are th points high
// (th = 32, or 64 for a single-iteration first pass) and T = 32 points wide.
struct LapOrigin {
    int u0, c0, x0, dlt;
};

__device__ __forceinline__ LapOrigin lap_origin(int W, int halo, int th, int tile) {
    const int tiles_x = div_up(W, T);
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    LapOrigin o;
    o.u0 = ty * th - halo;
    o.c0 = tx * T - halo;
    o.x0 = floor4(3 * o.c0);
    o.dlt = 3 * o.c0 - o.x0;
    return o;
}

// What a Laplacian tile needs, read from the frame's arguments once per tile: the batch kernel
// keeps them in global memory, where every barrier would make the compiler load them again.
struct LapJob {
    const float* points;
    const float* d_in;             // previous pass's displacement, or nullptr (first pass)
    float* d_out;
    float* export_points;
    int* error;
    int H, W, iters, halo, th;
    BoxGeom box;
    float lambda;
    LapOrigin og;
};

__device__ __forceinline__ LapJob lap_job(const FrameArgs& a, const LapPhase& ph, int tile) {
    LapJob j;
    j.points = a.points;
    j.d_in = ph.d_in;
    j.d_out = ph.d_out;
    j.export_points = ph.export_points;
    j.error = a.error;
    j.H = a.H;
    j.W = a.W;
    j.iters = ph.iters;
    j.halo = ph.halo;
    j.th = ph.tile_h;
    j.box = ph.box;
    j.lambda = a.lambda;
    j.og = lap_origin(j.W, j.halo, j.th, tile);
    return j;
}

// Issues the TMA load of a tile's box of input points into V0 (thread 0; completes on bar). The
// input points are never written inside the launch, so only the box's earlier shared-memory use
// needs ordering -- a global proxy fence would also wait for this thread's own pending stores.
__device__ __forceinline__ void lap_issue(const FrameArgs& a, const LapPhase& ph, const CUtensorMap* map, int tile,
                                          float* V0, uint64_t* bar) {
    if (threadIdx.x != 0) return;
    const LapOrigin o = lap_origin(a.W, ph.halo, ph.tile_h, tile);
    fence_proxy_async_shared();
    mbar_arrive_expect_tx(bar, (unsigned)(ph.box.rows * ph.box.cols * 4));
    tma_load_2d(V0, map, o.x0, o.u0, bar);
}
// One Jacobi iteration (Eq. 1-2) over the region [lo, RH - lo) x [lo, RW - lo) of the staged
// tile: from `cur` (displacements; unused when WITH_D = false) into `nxt`. A strip that runs
// past the region's last row computes its extra points from the box's spare rows and discards
// them; each kept point's window lies inside the region the previous iteration wrote.
template <int R, bool WITH_D>
__device__ __forceinline__ void lap_iteration(int H, int W, float lambda, int cols, const LapOrigin& og, int RH, int RW,
                                              int lo, const float* V0, const float* cur, float* nxt) {
    constexpr int S = kLapStrip;
    const int cw = RW - 2 * lo;
    const int strips = (RH - 2 * lo + S - 1) / S;
    // (strip, column) of item i = threadIdx.x + k blockDim.x, stepped without a division per item
    const int step_s = (int)blockDim.x / cw, step_c = (int)blockDim.x - step_s * cw;
    int sr = (int)threadIdx.x / cw, cc = (int)threadIdx.x - sr * cw;
    for (; sr < strips; sr += step_s, cc += step_c) {
        if (cc >= cw) {
            cc -= cw;
            ++sr;
            if (sr >= strips) break;
        }
        const int r = lo + S * sr, c = lo + cc;
        const int rows = min(S, RH - lo - r);
        const int o0 = r * cols + og.dlt + 3 * c;
        LapAcc A[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            A[k].c = lap_load<WITH_D>(V0, cur, o0 + k * cols);
            A[k].sx = A[k].sy = A[k].sz = A[k].ws = 0.f;
        }
        // Each point takes its window in row-major order whatever its place in the strip, so a
        // point's sum does not depend on how the strips fall (fused or split passes give the
        // same bits). Strip points m < k within the radius share one weight: computed when the
        // traversal reaches row m (where k needs it), kept for row k (where m needs it).
        float pex[S][S], pey[S][S], pez[S][S], pw[S][S];
#pragma unroll
        for (int dr = -R; dr < S + R; ++dr) {
#pragma unroll
            for (int dc = -R; dc <= R; ++dc) {
                if (dc == 0 && dr >= 0 && dr < S) {
                    const int m = dr;   // a strip point
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        if (k > m && k <= m + R) {
                            lap_diff<WITH_D>(A[m].c, A[k].c, pex[m][k], pey[m][k], pez[m][k]);
                            const float w = lap_weight(pex[m][k], pey[m][k], pez[m][k]);
                            pw[m][k] = w;
                            // fma(-w, e) = fma(w, -e): the same bits as k's own term for m
                            A[k].sx = fmaf(-w, pex[m][k], A[k].sx);
                            A[k].sy = fmaf(-w, pey[m][k], A[k].sy);
                            A[k].sz = fmaf(-w, pez[m][k], A[k].sz);
                            A[k].ws = __fadd_rn(A[k].ws, w);
                        }
                        if (k < m && k >= m - R)
                            lap_accumulate(A[k].sx, A[k].sy, A[k].sz, A[k].ws, pw[k][m], pex[k][m], pey[k][m],
                                           pez[k][m]);
                    }
                    continue;
                }
                const LapPt q = lap_load<WITH_D>(V0, cur, o0 + dr * cols + 3 * dc);
#pragma unroll
                for (int k = 0; k < S; ++k)
                    if (dr - k >= -R && dr - k <= R) lap_add<WITH_D>(A[k], q);
            }
        }
        // Eq. 1 on the displacement; the pinned border ring, invalid points and points without
        // a usable neighbour keep their displacement
        const int gu = og.u0 + r, gv = og.c0 + c;
        const bool colpin = gv < R || gv >= W - R;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            if (k >= rows) break;
            const bool keep = colpin || gu + k < R || gu + k >= H - R || A[k].c.x == kInvalidCoord || !(A[k].ws > 0.f);
            const float s = lap_scale(keep, lambda, A[k].ws);
            const int o = o0 + k * cols;
            nxt[o] = fmaf(s, A[k].sx, A[k].c.dx);
            nxt[o + 1] = fmaf(s, A[k].sy, A[k].c.dy);
            nxt[o + 2] = fmaf(s, A[k].sz, A[k].c.dz);
        }
    }
}

// One Laplacian tile: th x T output points, `iters` fused Jacobi iterations (Eq. 1-2). The input
// box is in V0, either already issued by TMA on `bar` (tma = true: wait for it) or to be loaded
// here with plain loads. Da, Db: the displacement ping-pong (a single-iteration first pass reads
// no displacement and writes only Db; then Da may alias Db). The box has kLapStrip - 1 spare rows
// below the tile's halo for the strips that run past the region.
template <int R>
__device__ void lap_tile(const LapJob& j, float* V0, float* Da, float* Db, bool tma, uint64_t* bar, unsigned parity) {
    const int H = j.H, W = j.W, h = j.halo, th = j.th;
    const int RH = th + 2 * h, RW = T + 2 * h;
    const BoxGeom b = j.box;                   // rows = RH + kLapStrip - 1, cols >= 3 RW + delta
    const LapOrigin og = j.og;
    const int u0 = og.u0, c0 = og.c0, dlt = og.dlt;
    const bool first = j.d_in == nullptr;

    if (!tma) stage_box(V0, j.points, nullptr, b, og.x0, u0, H, W, NAN, bar, 0, false);
    if (!first) stage_box(Da, j.d_in, nullptr, b, og.x0, u0, H, W, 0.f, bar, 0, false);
    if (tma) mbar_wait_bounded(bar, parity, j.error);   // the caller flips its parity
    __syncthreads();
    // invalid points (non-finite or out of range, including outside the image) become the
    // finite sentinel with zero displacement; the first pass reads no displacement, and without
    // iterations (lap_iters = 0) its output is the zero displacement itself
    const bool zero_all = first && j.iters == 0;
    // (row, column) of item i = threadIdx.x + k blockDim.x, stepped without a division per item;
    // four items per round, their loads issued together
    {
        constexpr int U = 4;
        const int step_r = blockDim.x / RW, step_c = blockDim.x - step_r * RW;
        int r = threadIdx.x / RW, c = threadIdx.x - r * RW;
        for (int i0 = threadIdx.x; i0 < RH * RW; i0 += U * blockDim.x) {
            int o[U];
            float x[U], y[U], z[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                o[u] = r * b.cols + dlt + 3 * c;
                r += step_r;
                c += step_c;
                if (c >= RW) {
                    c -= RW;
                    ++r;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool in = i0 + u * (int)blockDim.x < RH * RW;
                x[u] = in ? V0[o[u]] : 0.f;
                y[u] = in ? V0[o[u] + 1] : 0.f;
                z[u] = in ? V0[o[u] + 2] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (i0 + u * (int)blockDim.x >= RH * RW) break;
                const bool bad = !point_valid(x[u], y[u], z[u]);
                if (bad) V0[o[u]] = V0[o[u] + 1] = V0[o[u] + 2] = kInvalidCoord;
                if ((bad && !first) || zero_all) Da[o[u]] = Da[o[u] + 1] = Da[o[u] + 2] = 0.f;
            }
        }
    }
    __syncthreads();

    float* cur = Da;
    float* nxt = Db;
    for (int t = 1; t <= j.iters; ++t) {
        if (first && t == 1) lap_iteration<R, false>(H, W, j.lambda, b.cols, og, RH, RW, R, V0, cur, nxt);
        else lap_iteration<R, true>(H, W, j.lambda, b.cols, og, RH, RW, t * R, V0, cur, nxt);
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }

    // The tile's own points: displacement out (AoS, row-contiguous), optional export. With
    // W % 4 == 0 a tile row (96 floats) starts 16-byte aligned both here (dlt + 3h = 0 mod 4, the
    // box width a multiple of 4) and in the array (3W and 96 tx multiples of 4): float4 stores.
    if ((W & 3) == 0) {
        // thread -> tile rows threadIdx.x / 8 + 32 k and float4 columns (threadIdx.x % 8) + 8 m
        static_assert(kThreads == 8 * T && (3 * T / 4) % 8 == 0, "one tile row per 8 threads");
        const int q = threadIdx.x & 7;
        const int gv3 = 3 * (c0 + h) + 4 * q;
        for (int rr = threadIdx.x >> 3; rr < th; rr += kThreads / 8) {
            const int gu = u0 + h + rr;
            if (gu >= H) break;
            const float* src = cur + (h + rr) * b.cols + dlt + 3 * h + 4 * q;
            float* dst = j.d_out + (size_t)gu * 3 * W + gv3;
#pragma unroll
            for (int m = 0; m < 3 * T / 32; ++m)
                if (gv3 + 32 * m < 3 * W)   // then gv3 + 32 m + 3 < 3W as well
                    *reinterpret_cast<float4*>(dst + 32 * m) = *reinterpret_cast<const float4*>(src + 32 * m);
        }
    }
    if ((W & 3) != 0 || j.export_points) {
        for (int e = threadIdx.x; e < th * 3 * T; e += blockDim.x) {
            const int r = e / (3 * T), f = e - r * (3 * T);
            const int gu = u0 + h + r, gv3 = 3 * (c0 + h) + f;
            if (gu >= H || gv3 >= 3 * W) continue;
            const int o = (h + r) * b.cols + dlt + 3 * h + f;
            const size_t g = (size_t)gu * 3 * W + gv3;
            const float d = cur[o];
            if ((W & 3) != 0) j.d_out[g] = d;
            if (j.export_points) {
                const int pt = o - (f % 3);
                j.export_points[g] = V0[pt] != kInvalidCoord ? __fadd_rn(V0[o], d) : NAN;
            }
        }
    }
    __syncthreads();
}
// ------------------------------------------------------------------------------ bilateral

// A staged point: input position and displacement.
struct SP {
    float x, y, z, dx, dy, dz;
};

__device__ __forceinline__ SP load_sp(const float* V0, const float* D, int o) {
    return {V0[o], V0[o + 1], V0[o + 2], D[o], D[o + 1], D[o + 2]};
}

struct PairEdge {
    F2 x, y, z;
};

__device__ __forceinline__ PairEdge pair_edge(const SP& a, const SP& b) {
    return {pair_diff(a.x, a.dx, b.x, b.dx), pair_diff(a.y, a.dy, b.y, b.dy), pair_diff(a.z, a.dz, b.z, b.dz)};
}

__device__ __forceinline__ V3 pair_cross(const PairEdge& e1, const PairEdge& e2) {
    return {pair_sub_round(pair_mul(e1.y, e2.z), pair_mul(e1.z, e2.y)),
            pair_sub_round(pair_mul(e1.z, e2.x), pair_mul(e1.x, e2.z)),
            pair_sub_round(pair_mul(e1.x, e2.y), pair_mul(e1.y, e2.x))};
}

// Edge b - a in FP32 and the size of what was summed to form it (for the error bound).
struct FastEdge {
    V3 e;
    float m;    // sum over coordinates of the differences |v0_b - v0_a|, |d_b - d_a| that were rounded
    float l1;   // sum over coordinates of |e|
};

// |q - p| where the difference q - p was rounded, 0 where it is exact: a computed difference
// below both operands in magnitude proves that q lies within a factor 2 of p (rounding is
// monotonic, so the exact difference is below them too), and then q - p is exact (Sterbenz).
__device__ __forceinline__ float rounded_part(float diff, float p, float q) {
    const float ad = fabsf(diff);
    return ad < fminf(fabsf(p), fabsf(q)) ? 0.f : ad;
}

// Edge b - a in FP32 (the same value as fast_edge(a, b).e).
__device__ __forceinline__ V3 edge_of(const SP& a, const SP& b) {
    return {(b.x - a.x) + (b.dx - a.dx), (b.y - a.y) + (b.dy - a.dy), (b.z - a.z) + (b.dz - a.dz)};
}

// Dominant normals up to this count are held in registers by the group assignment.
constexpr int kRegGroups = 4;

__device__ __forceinline__ FastEdge fast_edge(const SP& a, const SP& b) {
    const float ax = b.x - a.x, ay = b.y - a.y, az = b.z - a.z;
    const float dx = b.dx - a.dx, dy = b.dy - a.dy, dz = b.dz - a.dz;
    FastEdge f;
    f.e = {ax + dx, ay + dy, az + dz};
    // (the displacements' differences are counted as rounded: they are rarely within a factor 2)
    f.m = (rounded_part(ax, a.x, b.x) + fabsf(dx)) + (rounded_part(ay, a.y, b.y) + fabsf(dy)) +
          (rounded_part(az, a.z, b.z) + fabsf(dz));
    f.l1 = fabsf(f.e.x) + fabsf(f.e.y) + fabsf(f.e.z);
    return f;
}

// Error of the FP32 normal. Each edge coordinate is off by at most u (m_c + |e_c|), u = 2^-24,
// m_c the rounded differences summed into it; the cross product adds u per product and u for
// the difference. So |d cr|_1 <= u (m1 |e2|_1 + |e1|_1 m2 + 4 |e1|_1 |e2|_1), and the angle is
// off by at most sqrt(3) |d cr|_1 / |cr|_1. Accept the FP32 normal when that bound is below
// sqrt(3) 64 u = 6.6e-6 rad (15 times inside the 1e-4 rad tolerance), otherwise recompute it
// from exact pairs.
__device__ __forceinline__ bool fast_cross_ok(const FastEdge& e1, const FastEdge& e2, V3 cr) {
    const float crl1 = fabsf(cr.x) + fabsf(cr.y) + fabsf(cr.z);
    return e1.m * e2.l1 + e1.l1 * e2.m + 4.f * (e1.l1 * e2.l1) <= 64.f * crl1;
}

__device__ __forceinline__ V3 centroid3(const SP& a, const SP& b, const SP& c) {
    const float k = 1.f / 3.f;
    return {((a.x + b.x + c.x) + (a.dx + b.dx + c.dx)) * k, ((a.y + b.y + c.y) + (a.dy + b.dy + c.dy)) * k,
            ((a.z + b.z + c.z) + (a.dz + b.dz + c.dz)) * k};
}

// Per-quad records in shared memory: 6 floats interleaving the quad's two triangles,
// {x0, x1, y0, y1, z0, z1}, so that each 64-bit load yields one coordinate of both triangles as
// a packed pair (f32x2.cuh).
__device__ __forceinline__ void load_quad(const float* A, int q, V3& t0, V3& t1) {
    const float2* p = reinterpret_cast<const float2*>(A) + 3 * q;
    const float2 x = p[0], y = p[1], z = p[2];
    t0 = {x.x, y.x, z.x};
    t1 = {x.y, y.y, z.y};
}

__device__ __forceinline__ void load_quad2(const float* A, int q, f2& x, f2& y, f2& z) {
    const f2* p = reinterpret_cast<const f2*>(A) + 3 * q;
    x = p[0];
    y = p[1];
    z = p[2];
}

__device__ __forceinline__ void store_quad(float* A, int q, V3 t0, V3 t1) {
    float2* p = reinterpret_cast<float2*>(A) + 3 * q;
    p[0] = make_float2(t0.x, t1.x);
    p[1] = make_float2(t0.y, t1.y);
    p[2] = make_float2(t0.z, t1.z);
}

__device__ __forceinline__ bool has_normal(V3 n) { return n.x != 0.f || n.y != 0.f || n.z != 0.f; }

__device__ __forceinline__ V3 finish_normal(V3 s, V3 own) {
    const float l2 = dot(s, s);
    if (!has_normal(own) || !(l2 > 0.f)) return own;
    const float inv = rsqrtf(l2);
    return {s.x * inv, s.y * inv, s.z * inv};
}

// One own triangle i against the two triangles of a neighbour quad at once, in packed pairs:
//   W_j = ex2(-(|c'_i - c'_j|^2 + a - a n_i . n_j)),   s_i += W_j n_j   (j = both triangles)
// The state holds i's centroid and -a n_i broadcast to both halves, and the two halves of the
// running sum (added together at the end).
struct OwnTri {
    f2 cx, cy, cz;
    f2 px, py, pz;
    f2 sx, sy, sz;
};

__device__ __forceinline__ void own_begin(OwnTri& o, V3 c, V3 n, float a) {
    o.cx = bc(c.x);
    o.cy = bc(c.y);
    o.cz = bc(c.z);
    o.px = bc(-a * n.x);
    o.py = bc(-a * n.y);
    o.pz = bc(-a * n.z);
    o.sx = o.sy = o.sz = 0ull;
}

__device__ __forceinline__ f2 own_weights(const OwnTri& o, f2 a2, f2 cx, f2 cy, f2 cz, f2 nx, f2 ny, f2 nz) {
    const f2 dx = sub2(o.cx, cx), dy = sub2(o.cy, cy), dz = sub2(o.cz, cz);
    f2 ne = fma2(o.px, nx, a2);
    ne = fma2(o.py, ny, ne);
    ne = fma2(o.pz, nz, ne);
    ne = fma2(dz, dz, ne);
    ne = fma2(dy, dy, ne);
    ne = fma2(dx, dx, ne);
    float e0, e1;
    upk(ne, e0, e1);
    return pk(ex2(-e0), ex2(-e1));
}

__device__ __forceinline__ void own_add(OwnTri& o, f2 w, f2 nx, f2 ny, f2 nz) {
    o.sx = fma2(w, nx, o.sx);
    o.sy = fma2(w, ny, o.sy);
    o.sz = fma2(w, nz, o.sz);
}

__device__ __forceinline__ V3 own_sum(const OwnTri& o) {
    float a, b, c, d, e, f;
    upk(o.sx, a, b);
    upk(o.sy, c, d);
    upk(o.sz, e, f);
    return {a + b, c + d, e + f};
}

// A quad's two triangles: their own quad first (each triangle's weight with itself is exactly 1).
struct QuadAcc {
    OwnTri t0, t1;
    V3 n0, n1;   // current normals (a triangle without a normal keeps n = 0)
};

__device__ __forceinline__ void quad_begin(QuadAcc& A, const float* Cq, const float* cur, int q, float a, f2 a2) {
    f2 cx, cy, cz, nx, ny, nz;
    load_quad2(Cq, q, cx, cy, cz);
    load_quad2(cur, q, nx, ny, nz);
    float c0x, c1x, c0y, c1y, c0z, c1z, n0x, n1x, n0y, n1y, n0z, n1z;
    upk(cx, c0x, c1x);
    upk(cy, c0y, c1y);
    upk(cz, c0z, c1z);
    upk(nx, n0x, n1x);
    upk(ny, n0y, n1y);
    upk(nz, n0z, n1z);
    A.n0 = {n0x, n0y, n0z};
    A.n1 = {n1x, n1y, n1z};
    own_begin(A.t0, {c0x, c0y, c0z}, A.n0, a);
    own_begin(A.t1, {c1x, c1y, c1z}, A.n1, a);
    const f2 w0 = own_weights(A.t0, a2, cx, cy, cz, nx, ny, nz);
    own_add(A.t0, pk(1.f, hi_of(w0)), nx, ny, nz);
    const f2 w1 = own_weights(A.t1, a2, cx, cy, cz, nx, ny, nz);
    own_add(A.t1, pk(lo_of(w1), 1.f), nx, ny, nz);
}

__device__ __forceinline__ void quad_neighbour(QuadAcc& A, f2 a2, f2 cx, f2 cy, f2 cz, f2 nx, f2 ny, f2 nz) {
    own_add(A.t0, own_weights(A.t0, a2, cx, cy, cz, nx, ny, nz), nx, ny, nz);
    own_add(A.t1, own_weights(A.t1, a2, cx, cy, cz, nx, ny, nz), nx, ny, nz);
}

// One bilateral tile: TH x T quads (TH = a.bil_th rows of T = 32, so that a warp spans a tile row);
// geometry, `ph.iters` fused iterations (Eq. 3-6), then either
// the carry for the next chunk or mask, normals, groups (Algorithm 4) and the tile-local
// segments (Algorithm 5); with JOIN (the single-frame kernel) also the joins across the tile's
// borders with finished neighbours.
// Shared-memory header of the persistent kernels (128 bytes before the tiles' buffers): the staging
// mbarriers from byte 0, the bilateral tile's deferred-normal count at byte 64, and for the stage
// timing the last stamp at byte 72 and the stage totals' address (or nullptr) at byte 80.
constexpr int kHdrExact = 64, kHdrStamp = 72, kHdrStages = 80;

// The borders of a finished tile's segments with its neighbours' (defined with the merge phase).
__device__ __forceinline__ void join_tile_borders(const FrameArgs& a, int tile);

__device__ __forceinline__ void set_stage_timing(uint64_t* bar, unsigned long long* sns) {
    if (threadIdx.x == 0) *reinterpret_cast<unsigned long long**>(reinterpret_cast<unsigned char*>(bar) + kHdrStages) = sns;
}

// With stage timing on (set_stage_timing), thread 0 adds the tile's time in each stage -- staging,
// geometry, iterations, finish (groups and outputs, or the carry), tile labels -- to the totals
// (%globaltimer nanoseconds summed over tiles: CTA time, not wall time). The state lives in the
// shared-memory header, so that it holds no register across the tile.
__device__ __forceinline__ void stage_mark(uint64_t* bar, int k) {
    if (threadIdx.x == 0) {
        unsigned char* hdr = reinterpret_cast<unsigned char*>(bar);
        unsigned long long* sns = *reinterpret_cast<unsigned long long**>(hdr + kHdrStages);
        if (sns) {
            unsigned long long* last = reinterpret_cast<unsigned long long*>(hdr + kHdrStamp);
            const unsigned long long t = global_ns();
            if (k >= 0) atomicAdd(sns + k, t - *last);
            *last = t;
        }
    }
}

template <int R, bool JOIN>
__device__ void bil_tile(const FrameArgs& a, const BilPhase& ph, int tile, float* smem, uint64_t* bar,
                         unsigned& parity) {
    stage_mark(bar, -1);
    // the frame's arguments, read once (the batch kernel keeps them in global memory, where every
    // barrier and every global store would make the compiler load them again)
    const int H = a.H, W = a.W, Hq = H - 1, Wq = W - 1;
    const int h = ph.halo, iters = ph.iters;
    const bool first = ph.first != 0, last = ph.last != 0;
    const float* const carry_in = ph.carry_in;
    float* const carry_out = ph.carry_out;
    int* const error = a.error;
    const float max_edge2 = a.max_edge2;
    const int TH = a.bil_th;
    const int RQH = TH + 2 * h, RQW = T + 2 * h;         // staged quads
    const int nq = RQH * RQW;
    const int nqs = nq + RQW;                            // one spare row of quads
    const BoxGeom b = ph.box;                            // rows = RQH + 1 points, cols >= 3 (RQW + 1) + delta
    const int bsz = align_floats(b.rows * b.cols);
    float* Cq = smem;                                    // [nqs][6] scaled centroids
    float* Na = Cq + align_floats(6 * nqs);              // [nqs][6] normals
    float* X = Na + align_floats(6 * nqs);               // Nb, or the two staged boxes before the iterations
    float* Nb = X;
    float* V0 = X;
    float* Dp = X + bsz;
    const int xw = max(align_floats(6 * nqs), 2 * bsz);
    uint8_t* Mk = reinterpret_cast<uint8_t*>(X + xw);    // [TH*T*2] own masks (room for T*T*2)
    uint8_t* Gs = Mk + 2 * T * T;                        // [TH*T*2] own groups
    int* ex_list = reinterpret_cast<int*>(Gs + 2 * T * T);   // [kExactCap] deferred exact normals
    const int tiles_x = div_up(Wq, T);
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int qu0 = ty * TH - h, qv0 = tx * T - h;
    const int x0 = floor4(3 * qv0);
    const int dlt = 3 * qv0 - x0;
    const float cs = a.c_scale;

    const CUtensorMap* mp = ph.use_tma ? &a.tm_pts_bil : nullptr;
    const CUtensorMap* md = ph.use_tma ? &a.tm_disp_bil : nullptr;
    if (mp && threadIdx.x == 0) fence_proxy_async_all();
    stage_box(V0, a.points, mp, b, x0, qu0, H, W, NAN, bar, 2, true);
    stage_box(Dp, a.disp, md, b, x0, qu0, H, W, 0.f, bar, 0, true);
    if (mp) {
        mbar_wait_bounded(bar, parity, error);
        parity ^= 1u;
    }
    __syncthreads();
    int* n_exact = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(bar) + kHdrExact);   // in the smem header
    if (threadIdx.x == 0) *n_exact = 0;
    {
        // (row, column) of point i = threadIdx.x + k blockDim.x, stepped without a division; four
        // points per round, their loads issued together
        constexpr int U = 4;
        const int PW = RQW + 1, NP = (RQH + 1) * PW;
        const int step_r = blockDim.x / PW, step_c = blockDim.x - step_r * PW;
        int r = threadIdx.x / PW, c = threadIdx.x - r * PW;
        for (int i0 = threadIdx.x; i0 < NP; i0 += U * blockDim.x) {
            int o[U];
            float x[U], y[U], z[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                o[u] = r * b.cols + dlt + 3 * c;
                r += step_r;
                c += step_c;
                if (c >= PW) {
                    c -= PW;
                    ++r;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool in = i0 + u * (int)blockDim.x < NP;
                x[u] = in ? V0[o[u]] : 0.f;
                y[u] = in ? V0[o[u] + 1] : 0.f;
                z[u] = in ? V0[o[u] + 2] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (i0 + u * (int)blockDim.x >= NP) break;
                if (!point_valid(x[u], y[u], z[u])) {
                    V0[o[u]] = V0[o[u] + 1] = V0[o[u] + 2] = NAN;
                    Dp[o[u]] = Dp[o[u] + 1] = Dp[o[u] + 2] = 0.f;
                }
            }
        }
    }
    __syncthreads();
    stage_mark(bar, 0);

    // Centroids and normals of every staged triangle; masks of the tile's own quads. A normal
    // whose FP32 error bound fails is deferred: its quad goes on a short list that a second
    // loop recomputes from exact pairs with every lane busy (inline, divergent, only when the
    // list is full).
    auto exact_normals = [&](const SP& p1, const SP& p2, const SP& p3, const SP& p4, bool do0, bool do1, V3& n0,
                             V3& n1) {
        const PairEdge pd = pair_edge(p3, p1);
        if (do0) n0 = pair_cross(pair_edge(p3, p2), pd);
        if (do1) {
            const PairEdge pdn = {{-pd.x.h, -pd.x.l}, {-pd.y.h, -pd.y.l}, {-pd.z.h, -pd.z.l}};
            n1 = pair_cross(pair_edge(p1, p4), pdn);
        }
    };
    auto unit_or_none = [](V3 cr, bool valid) {
        const float len2 = dot(cr, cr);
        V3 n = {0.f, 0.f, 0.f};
        if (valid && len2 > kDegenerateLen2) {
            const float inv = rsqrtf(len2);
            n = {cr.x * inv, cr.y * inv, cr.z * inv};
        }
        return n;
    };
    auto scaled_centroid = [&](const SP& va, const SP& vb, const SP& vc, V3 n) {
        V3 c = {kAbsentCentroid, kAbsentCentroid, kAbsentCentroid};
        if (has_normal(n)) {
            const V3 m = centroid3(va, vb, vc);
            c = {m.x * cs, m.y * cs, m.z * cs};
        }
        return c;
    };
    // (row, column) of quad q = threadIdx.x + k blockDim.x, stepped without a division per quad
    const int gstep_r = blockDim.x / RQW, gstep_c = blockDim.x - gstep_r * RQW;
    int g_qr = threadIdx.x / RQW, g_qc = threadIdx.x - g_qr * RQW;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int qr = g_qr, qc = g_qc;
        g_qr += gstep_r;
        g_qc += gstep_c;
        if (g_qc >= RQW) {
            g_qc -= RQW;
            ++g_qr;
        }
        const int gu = qu0 + qr, gv = qv0 + qc;
        const bool exists = gu >= 0 && gu < Hq && gv >= 0 && gv < Wq;
        const int o1 = qr * b.cols + dlt + 3 * qc;
        const SP p1 = load_sp(V0, Dp, o1), p2 = load_sp(V0, Dp, o1 + 3);
        const SP p3 = load_sp(V0, Dp, o1 + b.cols + 3), p4 = load_sp(V0, Dp, o1 + b.cols);
        const bool own = last && qr >= h && qr < h + TH && qc >= h && qc < h + T;
        const bool v1 = p1.x == p1.x, v2 = p2.x == p2.x, v3 = p3.x == p3.x, v4 = p4.x == p4.x;
        const bool valid0 = exists && v1 && v2 && v3;                            // Algorithm 1
        const bool valid1 = exists && v1 && v3 && v4;
        V3 nn[2] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        // first = {p3, p2, p1}: (p2 - p3) x (p1 - p3);  second = {p1, p4, p3}: (p4 - p1) x (p3 - p1)
        const FastEdge er = fast_edge(p3, p2), ed = fast_edge(p3, p1), el = fast_edge(p1, p4);
        if (first) {
            const FastEdge edn = {{-ed.e.x, -ed.e.y, -ed.e.z}, ed.m, ed.l1};
            V3 cr0 = cross(er.e, ed.e), cr1 = cross(el.e, edn.e);
            const bool exact0 = valid0 && !fast_cross_ok(er, ed, cr0);
            const bool exact1 = valid1 && !fast_cross_ok(el, edn, cr1);
            bool defer = false;
            if (exact0 || exact1) {
                const int slot = atomicAdd(n_exact, 1);
                if (slot < kExactCap) {
                    ex_list[slot] = q | (exact0 ? 1 << 29 : 0) | (exact1 ? 1 << 30 : 0);
                    defer = true;
                } else {
                    exact_normals(p1, p2, p3, p4, exact0, exact1, cr0, cr1);
                }
            }
            // a deferred quad's records are written again by the second loop
            nn[0] = unit_or_none(cr0, valid0 && !(defer && exact0));
            nn[1] = unit_or_none(cr1, valid1 && !(defer && exact1));
        } else {
            const bool vk[2] = {valid0, valid1};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!vk[k]) continue;
                const size_t gid = 2 * ((size_t)gu * Wq + gv) + k;
                const float nx = __ldcg(carry_in + 3 * gid);   // written by the previous pass
                if (nx == nx) nn[k] = {nx, __ldcg(carry_in + 3 * gid + 1), __ldcg(carry_in + 3 * gid + 2)};
            }
        }
        const V3 cc0 = scaled_centroid(p3, p2, p1, nn[0]), cc1 = scaled_centroid(p1, p4, p3, nn[1]);
        if (own) {                                                               // Algorithm 4, l_max
            // FP32 edges: ~1e-7 relative error, far inside the 1e-5 m band where FP32 and FP64
            // may disagree
            const V3 et = edge_of(p2, p1), eb = edge_of(p4, p3);
            const float d2 = dot(ed.e, ed.e);
            const float l0 = fmaxf(d2, fmaxf(dot(er.e, er.e), dot(et, et)));
            const float l1 = fmaxf(d2, fmaxf(dot(el.e, el.e), dot(eb, eb)));
            const int t = 2 * ((qr - h) * T + (qc - h));
            Mk[t] = (valid0 && l0 <= max_edge2) ? 1 : 0;
            Mk[t + 1] = (valid1 && l1 <= max_edge2) ? 1 : 0;
        }
        store_quad(Cq, q, cc0, cc1);
        store_quad(Na, q, nn[0], nn[1]);
    }
    __syncthreads();
    // the deferred normals (and their centroids), one quad per lane
    const int n_ex = min(*n_exact, kExactCap);
    for (int i = threadIdx.x; i < n_ex; i += blockDim.x) {
        const int e = ex_list[i];
        const int q = e & ((1 << 29) - 1);
        const bool do0 = (e >> 29) & 1, do1 = (e >> 30) & 1;
        const int qr = q / RQW, qc = q - qr * RQW;
        const int o1 = qr * b.cols + dlt + 3 * qc;
        const SP p1 = load_sp(V0, Dp, o1), p2 = load_sp(V0, Dp, o1 + 3);
        const SP p3 = load_sp(V0, Dp, o1 + b.cols + 3), p4 = load_sp(V0, Dp, o1 + b.cols);
        V3 cr0 = {0.f, 0.f, 0.f}, cr1 = cr0;
        exact_normals(p1, p2, p3, p4, do0, do1, cr0, cr1);
        // the flagged triangles are valid (the flag requires it); write only their slots
        float* cq = Cq + 6 * q;
        float* na = Na + 6 * q;
        if (do0) {
            const V3 n = unit_or_none(cr0, true), c = scaled_centroid(p3, p2, p1, n);
            na[0] = n.x, na[2] = n.y, na[4] = n.z;
            cq[0] = c.x, cq[2] = c.y, cq[4] = c.z;
        }
        if (do1) {
            const V3 n = unit_or_none(cr1, true), c = scaled_centroid(p1, p4, p3, n);
            na[1] = n.x, na[3] = n.y, na[5] = n.z;
            cq[1] = c.x, cq[3] = c.y, cq[5] = c.z;
        }
    }
    __syncthreads();   // the staged boxes are dead from here on; Nb reuses their space
    stage_mark(bar, 1);

    // Fused bilateral iterations: each work item is a vertical pair of quads.
    float* cur = Na;
    float* nxt = Nb;
    const float an = a.a_norm;
    const f2 a2 = bc(an);
    for (int it = 1; it <= iters; ++it) {
        const int lo = it * R;
        const int ch = RQH - 2 * lo, cw = RQW - 2 * lo;
        const int strips = (ch + 1) >> 1;
        for (int i = threadIdx.x; i < strips * cw; i += blockDim.x) {
            const int sr = i / cw;
            const int qr = lo + 2 * sr, qc = lo + (i - sr * cw);
            const bool two = qr + 1 < RQH - lo;
            const int qA = qr * RQW + qc, qB = qA + RQW;
            QuadAcc A, B;
            quad_begin(A, Cq, cur, qA, an, a2);
            quad_begin(B, Cq, cur, qB, an, a2);
#pragma unroll
            for (int dr = -R; dr <= R + 1; ++dr) {
#pragma unroll
                for (int dc = -R; dc <= R; ++dc) {
                    const bool forA = dr <= R && !(dr == 0 && dc == 0);
                    const bool forB = dr >= 1 - R && !(dr == 1 && dc == 0);
                    const int qj = qA + dr * RQW + dc;
                    f2 cx, cy, cz, nx, ny, nz;
                    load_quad2(Cq, qj, cx, cy, cz);
                    load_quad2(cur, qj, nx, ny, nz);
                    if (forA) quad_neighbour(A, a2, cx, cy, cz, nx, ny, nz);
                    if (forB) quad_neighbour(B, a2, cx, cy, cz, nx, ny, nz);
                }
            }
            store_quad(nxt, qA, finish_normal(own_sum(A.t0), A.n0), finish_normal(own_sum(A.t1), A.n1));
            if (two) store_quad(nxt, qB, finish_normal(own_sum(B.t0), B.n0), finish_normal(own_sum(B.t1), B.n1));
        }
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    stage_mark(bar, 2);

    if (!last) {
        for (int i = threadIdx.x; i < TH * T; i += blockDim.x) {
            const int r = i / T, c = i - r * T;
            const int gu = ty * TH + r, gv = tx * T + c;
            if (gu >= Hq || gv >= Wq) continue;
            V3 n[2];
            load_quad(cur, (r + h) * RQW + (c + h), n[0], n[1]);
            const size_t gid0 = 2 * ((size_t)gu * Wq + gv);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const bool has = has_normal(n[k]);
                float* o = carry_out + 3 * (gid0 + k);
                o[0] = has ? n[k].x : NAN;
                o[1] = has ? n[k].y : NAN;
                o[2] = has ? n[k].z : NAN;
            }
        }
        __syncthreads();
        stage_mark(bar, 3);
        return;
    }

    // free after the last iteration (>= 6 * nqs floats, nqs >= (TH + 1) T): union-find parents, the
    // run representative of each triangle, and the tile root of each representative [TH*T*2] each
    int32_t* Lp = reinterpret_cast<int32_t*>(nxt);
    int32_t* RunOf = Lp + 2 * TH * T;
    int32_t* RootOf = RunOf + 2 * TH * T;
    uint8_t* const out_mask = a.out_mask;
    float* const out_normals = a.out_normals;
    uint8_t* const out_groups = a.groups;
    int32_t* const sizes = a.sizes;
    const float min_dot = a.min_dot;
    // up to kRegGroups dominant normals held in registers; more are read from the arguments
    const int K = a.nd.K;
    const float* const ndv = a.nd.v;
    float nd[3 * kRegGroups];
#pragma unroll
    for (int j = 0; j < 3 * kRegGroups; ++j) nd[j] = j < 3 * K ? ndv[j] : 0.f;
    // quads' outputs as 2-byte and 8-byte stores when the arrays allow (a quad starts at an even
    // GID; sizes, when present, are scratch of this library and 8-byte aligned)
    const bool vec_out = ((uintptr_t)out_mask & 1u) == 0 && ((uintptr_t)out_groups & 1u) == 0 &&
                         ((uintptr_t)out_normals & 7u) == 0;
    for (int i = threadIdx.x; i < TH * T; i += blockDim.x) {
        const int r = i / T, c = i - r * T;
        const int gu = ty * TH + r, gv = tx * T + c;
        const bool exists = gu < Hq && gv < Wq;
        V3 n[2];
        load_quad(cur, (r + h) * RQW + (c + h), n[0], n[1]);
        const size_t gid0 = exists ? 2 * ((size_t)gu * Wq + gv) : 0;
        int gk[2];
        bool kk[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int t = 2 * i + k;
            const bool kept = Mk[t] != 0;
            const bool has = has_normal(n[k]);
            int g = PL3D_NO_GROUP;
            if (exists && kept && has) {                                         // Algorithm 4, ang_min
                float best = -1.0f;
                if (K <= kRegGroups) {
#pragma unroll
                    for (int j = 0; j < kRegGroups; ++j) {
                        if (j >= K) break;
                        const float s = n[k].x * nd[3 * j] + n[k].y * nd[3 * j + 1] + n[k].z * nd[3 * j + 2];
                        if (s > best) {
                            best = s;
                            g = j;
                        }
                    }
                } else {
                    for (int j = 0; j < K; ++j) {
                        const float s = n[k].x * ndv[3 * j] + n[k].y * ndv[3 * j + 1] + n[k].z * ndv[3 * j + 2];
                        if (s > best) {
                            best = s;
                            g = j;
                        }
                    }
                }
                if (best < min_dot) g = PL3D_NO_GROUP;
            }
            gk[k] = g;
            kk[k] = kept;
            if (!has) n[k] = {NAN, NAN, NAN};
            Gs[t] = exists ? (uint8_t)g : (uint8_t)PL3D_NO_GROUP;
        }
        if (exists) {
            // the quad's two triangles are consecutive GIDs: one store per array when aligned
            if (vec_out) {
                *reinterpret_cast<uint16_t*>(out_mask + gid0) = (uint16_t)((kk[0] ? 1 : 0) | (kk[1] ? 256 : 0));
                *reinterpret_cast<uint16_t*>(out_groups + gid0) = (uint16_t)(gk[0] | (gk[1] << 8));
                float2* o = reinterpret_cast<float2*>(out_normals + 3 * gid0);
                o[0] = make_float2(n[0].x, n[0].y);
                o[1] = make_float2(n[0].z, n[1].x);
                o[2] = make_float2(n[1].y, n[1].z);
            } else {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    out_mask[gid0 + k] = kk[k] ? 1 : 0;
                    out_groups[gid0 + k] = (uint8_t)gk[k];
                    float* o = out_normals + 3 * (gid0 + k);
                    o[0] = n[k].x;
                    o[1] = n[k].y;
                    o[2] = n[k].z;
                }
            }
            if (sizes) *reinterpret_cast<int2*>(sizes + gid0) = make_int2(0, 0);
        }
    }
    __syncthreads();
    stage_mark(bar, 3);

    // Connected components inside the tile (twins of Algorithm 2 that stay in the tile).
    const bool offs = a.max_offset_scaled > 0.f;
    const float lim = a.max_offset_scaled;
    auto offset_ok = [&](int g, V3 ci, V3 cj) {
        const float* n = ndv + 3 * g;
        return !offs || fabsf(n[0] * (ci.x - cj.x) + n[1] * (ci.y - cj.y) + n[2] * (ci.z - cj.z)) <= lim;
    };
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // (1) Runs along each quad row. Chain position 2v is second(v), 2v+1 is first(v).
    for (int r = warp; r < TH; r += kThreads / 32) {
        const int tf = 2 * (r * T + lane), ts = tf + 1;
        const int gf = Gs[tf], gs = Gs[ts];
        V3 cf = {0.f, 0.f, 0.f}, cs2 = cf;
        if (offs) load_quad(Cq, (r + h) * RQW + (lane + h), cf, cs2);
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
            const int t0 = 2 * (r * T + l0);
            return ((p & 1) || !((brk_f_mask >> l0) & 1u)) ? t0 : t0 + 1;
        };
        const int rep_s = gs != PL3D_NO_GROUP ? root_of(start_s) : -1;
        const int rep_f = gf != PL3D_NO_GROUP ? root_of(start_f) : -1;
        Lp[ts] = rep_s;
        Lp[tf] = rep_f;
        RunOf[ts] = rep_s;
        RunOf[tf] = rep_f;
    }
    __syncthreads();
    // (2) Rows joined across horizontal edges: first(r, v) with second(r-1, v); one union per
    // run pair (a lane skips the pair its left neighbour already joined). Each warp takes a block
    // of consecutive edges, top down, so that a union finds the row above already joined and the
    // trees stay shallow (rows dealt to the warps in turn left chains as long as the tile is high;
    // the tile's label stage took 9.6 us instead of 7.5 us on the 480x640 frame).
    const int per_w = (TH - 1 + kThreads / 32 - 1) / (kThreads / 32);
    for (int r = 1 + warp * per_w, r_end = min(TH, 1 + (warp + 1) * per_w); r < r_end; ++r) {
        const int tf = 2 * (r * T + lane), tu = 2 * ((r - 1) * T + lane) + 1;
        const int gf = Gs[tf];
        bool link = gf != PL3D_NO_GROUP && Gs[tu] == gf;
        if (offs && link) {
            V3 cf, c1, c0u, cu;
            load_quad(Cq, (r + h) * RQW + (lane + h), cf, c1);
            load_quad(Cq, (r - 1 + h) * RQW + (lane + h), c0u, cu);
            link = offset_ok(gf, cf, cu);
        }
        const int ra = link ? RunOf[tf] : -1, rb = link ? RunOf[tu] : -1;
        const int pa = __shfl_up_sync(kFull, ra, 1), pb = __shfl_up_sync(kFull, rb, 1);
        const bool dup = lane > 0 && pa == ra && pb == rb;
        if (link && !dup) uf_unite(Lp, ra, rb);
    }
    __syncthreads();
    // (3) Only the run representatives were linked by the unions: each finds its root, halving
    // the path as it walks (concurrent walks only shorten paths, so they stay valid).
    for (int t = threadIdx.x; t < 2 * TH * T; t += blockDim.x)
        if (RunOf[t] == t) RootOf[t] = uf_find(Lp, t);
    __syncthreads();
    // (4) Each triangle leaves with the GID of its tile-local root (-1 without a group).
    int32_t* const labels = a.labels;
    const bool vec_lab = ((uintptr_t)labels & 7u) == 0;   // a quad's two labels in one 8-byte store
    for (int i = threadIdx.x; i < TH * T; i += blockDim.x) {
        const int r = i / T, c = i - r * T;
        const int gu = ty * TH + r, gv = tx * T + c;
        if (gu >= Hq || gv >= Wq) continue;
        const size_t gid0 = 2 * ((size_t)gu * Wq + gv);
        int lab[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int rep = RunOf[2 * i + k];
            lab[k] = -1;
            if (rep >= 0) {
                const int root = RootOf[rep];
                const int rq = root >> 1, rr = rq / T, rc = rq - rr * T;
                lab[k] = (int)(2 * ((size_t)(ty * TH + rr) * Wq + (tx * T + rc)) + (root & 1));
            }
        }
        if (vec_lab) {
            *reinterpret_cast<int2*>(labels + gid0) = make_int2(lab[0], lab[1]);
        } else {
            labels[gid0] = lab[0];
            labels[gid0 + 1] = lab[1];
        }
    }
    __syncthreads();
    // (5) The borders with the neighbouring tiles, when this launch joins them here (the
    // single-frame kernel; the batch kernel joins them in its merge phase).
    if (JOIN && a.border) join_tile_borders(a, tile);
    stage_mark(bar, 4);
}

// ------------------------------------------------------------------------- segments (Alg. 5)

// Centroid of triangle k of quad (u, v) from the smoothed points v0 + d (offset test only).
__device__ __forceinline__ V3 centroid_global(const FrameArgs& a, int u, int v, int k) {
    const int W = a.W;
    const size_t p1 = (size_t)u * W + v, p2 = p1 + 1, p3 = p1 + W + 1, p4 = p1 + W;
    const size_t ia = 3 * (k == 0 ? p3 : p1), ib = 3 * (k == 0 ? p2 : p4), ic = 3 * (k == 0 ? p1 : p3);
    const float* P = a.points;
    const float* D = a.disp;   // written earlier in this launch: L2-coherent loads
    const float kk = 1.f / 3.f;
    return {((P[ia] + P[ib] + P[ic]) + (__ldcg(D + ia) + __ldcg(D + ib) + __ldcg(D + ic))) * kk,
            ((P[ia + 1] + P[ib + 1] + P[ic + 1]) + (__ldcg(D + ia + 1) + __ldcg(D + ib + 1) + __ldcg(D + ic + 1))) * kk,
            ((P[ia + 2] + P[ib + 2] + P[ic + 2]) + (__ldcg(D + ia + 2) + __ldcg(D + ib + 2) + __ldcg(D + ic + 2))) * kk};
}

// Twins that cross a tile border: the top edge of a tile's first quad row and the right edge of
// its last quad column (tiles of a.bil_th x T quads). Work items: (row borders) x Wq, then
// (column borders) x Hq. Returns
// whether item w joins two triangles, and then their current labels (each in its triangle's
// set: the tile root, or an ancestor of it once a union has linked that root).
__device__ __forceinline__ bool merge_pair(const FrameArgs& a, long long w, int& ra, int& rb) {
    const int Wq = a.W - 1, Hq = a.H - 1, TH = a.bil_th;
    const long long n_row_items = (long long)(div_up(Hq, TH) - 1) * Wq;
    int u, v, uj, vj;
    if (w < n_row_items) {
        u = (int)(w / Wq + 1) * TH;
        v = (int)(w % Wq);
        uj = u - 1;
        vj = v;
    } else {
        const long long x = w - n_row_items;
        v = (int)(x / Hq + 1) * T - 1;
        u = (int)(x % Hq);
        uj = u;
        vj = v + 1;
    }
    const int i = 2 * (u * Wq + v);
    const int j = 2 * (uj * Wq + vj) + 1;
    const int g = __ldcg(a.groups + i);   // written by the bilateral pass of this launch
    if (g == PL3D_NO_GROUP || __ldcg(a.groups + j) != g) return false;
    if (a.max_offset > 0.f) {
        const V3 ci = centroid_global(a, u, v, 0), cj = centroid_global(a, uj, vj, 1);
        const float* nd = a.nd.v + 3 * g;
        if (fabsf(nd[0] * (ci.x - cj.x) + nd[1] * (ci.y - cj.y) + nd[2] * (ci.z - cj.z)) > a.max_offset) return false;
    }
    ra = __ldcg(a.labels + i);
    rb = __ldcg(a.labels + j);
    return true;
}

// merge_pair with the item's two groups and two labels loaded together (one round trip to L2
// instead of two; the labels are read whether or not the item joins).
__device__ __forceinline__ bool merge_pair_eager(const FrameArgs& a, long long w, int& ra, int& rb) {
    const int Wq = a.W - 1, Hq = a.H - 1, TH = a.bil_th;
    const long long n_row_items = (long long)(div_up(Hq, TH) - 1) * Wq;
    int u, v, uj, vj;
    if (w < n_row_items) {
        u = (int)(w / Wq + 1) * TH;
        v = (int)(w % Wq);
        uj = u - 1;
        vj = v;
    } else {
        const long long x = w - n_row_items;
        v = (int)(x / Hq + 1) * T - 1;
        u = (int)(x % Hq);
        uj = u;
        vj = v + 1;
    }
    const int i = 2 * (u * Wq + v);
    const int j = 2 * (uj * Wq + vj) + 1;
    const int g = __ldcg(a.groups + i), gj = __ldcg(a.groups + j);
    ra = __ldcg(a.labels + i);
    rb = __ldcg(a.labels + j);
    if (g == PL3D_NO_GROUP || gj != g) return false;
    if (a.max_offset > 0.f) {
        const V3 ci = centroid_global(a, u, v, 0), cj = centroid_global(a, uj, vj, 1);
        const float* nd = a.nd.v + 3 * g;
        if (fabsf(nd[0] * (ci.x - cj.x) + nd[1] * (ci.y - cj.y) + nd[2] * (ci.z - cj.z)) > a.max_offset) return false;
    }
    return true;
}

// One union per distinct pair in a warp: consecutive lanes walk one border, where long runs
// of twins join the same two tile segments; a lane whose pair (and frame) equals its left
// neighbour's leaves the union to that lane. Called by whole warps.
__device__ __forceinline__ void merge_unite(int32_t* labels, bool link, int ra, int rb, int frame) {
    if (!link) ra = rb = -1;
    const int pa = __shfl_up_sync(0xffffffffu, ra, 1), pb = __shfl_up_sync(0xffffffffu, rb, 1);
    const int pf = __shfl_up_sync(0xffffffffu, frame, 1);
    const bool dup = (threadIdx.x & 31) > 0 && pa == ra && pb == rb && pf == frame;
    if (link && !dup) uf_unite(labels, ra, rb);
}

// Joins a finished tile's segments with its neighbours' across the tile's borders, in the
// bilateral pass instead of a merge phase of its own. Each border is joined by the second of its
// two tiles to finish: both add 1 to the border's counter (an acquire-release atomic, after the
// barrier that ends the tile's label stores), and the one that reads an odd count joins it, so
// that no tile waits for another. Every launch adds 2 to each counter, so the counters are even
// between launches. Counter 2t is tile t's top border, 2t + 1 its left border. Warp k of the CTA
// takes side k (top, left, bottom, right), its lanes along the border (merge_pair's items); the
// other warps go on. Each item's groups and labels are loaded together; the unions halve the
// paths they walk, which keeps the trees shallow for the flatten phase (walking both paths side by
// side without halving measured 6 us slower per 480x640 frame, most of it in the flatten).
__device__ __forceinline__ void join_tile_borders(const FrameArgs& a, int tile) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= 4) return;
    const int Wq = a.W - 1, Hq = a.H - 1, TH = a.bil_th;
    const int tiles_x = div_up(Wq, T), tiles_y = div_up(Hq, TH);
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const bool has = warp == 0 ? ty > 0 : warp == 1 ? tx > 0 : warp == 2 ? ty + 1 < tiles_y : tx + 1 < tiles_x;
    if (!has) return;
    const int c = warp == 0 ? 2 * tile : warp == 1 ? 2 * tile + 1 : warp == 2 ? 2 * (tile + tiles_x) : 2 * (tile + 1) + 1;
    unsigned n = 0;
    if (lane == 0) n = atom_add_acq_rel_gpu(a.border + c, 1u);
    __syncwarp();   // the lanes' loads below ordered after lane 0's acquire
    if (!(__shfl_sync(0xffffffffu, n, 0) & 1u)) return;   // the neighbour joins it when it finishes
    // row borders first among the items, then columns
    const long long n_row_items = (long long)(tiles_y - 1) * Wq;
    const int len = (warp & 1) ? min(TH, Hq - ty * TH) : min(T, Wq - tx * T);
    const long long w0 = warp == 0   ? (long long)(ty - 1) * Wq + tx * T
                         : warp == 1 ? n_row_items + (long long)(tx - 1) * Hq + ty * TH
                         : warp == 2 ? (long long)ty * Wq + tx * T
                                     : n_row_items + (long long)tx * Hq + ty * TH;
    int32_t* const L = a.labels;
    for (int i0 = 0; i0 < len; i0 += 32) {   // the same trip count in every lane
        int ra = -1, rb = -1;
        const bool link = i0 + lane < len && merge_pair_eager(a, w0 + i0 + lane, ra, rb);
        if (!link) ra = rb = -1;
        const int pa = __shfl_up_sync(0xffffffffu, ra, 1), pb = __shfl_up_sync(0xffffffffu, rb, 1);
        const bool dup = lane > 0 && pa == ra && pb == rb;   // one union per distinct pair
        if (link && !dup) uf_unite(L, ra, rb);
    }
}

__device__ __forceinline__ void merge_phase(const FrameArgs& a) {
    const int Wq = a.W - 1, Hq = a.H - 1;
    const long long n = (long long)(div_up(Hq, a.bil_th) - 1) * Wq + (long long)(div_up(Wq, T) - 1) * Hq;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_iter = (n + stride - 1) / stride;   // uniform: whole warps stay together
    const long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long it = 0; it < n_iter; ++it) {
        const long long w = base + it * stride;
        int ra = -1, rb = -1;
        const bool link = w < n && merge_pair(a, w, ra, rb);
        merge_unite(a.labels, link, ra, rb, 0);
    }
}

// Root of a label whose parent has already been loaded (no union runs any more; L2 loads, as
// other threads overwrite labels with roots meanwhile -- an ancestor either way).
__device__ __forceinline__ int root_from(const int32_t* L, int x, int p) {
    while (p != x) {
        x = p;
        p = __ldcg(L + x);
    }
    return x;
}

// Every grouped triangle takes its root; with tri_min > 0 the segment sizes are counted, one
// atomic per run of equal roots in a warp. Four triangles per thread are in flight at once:
// their labels, then their parents, are loaded together before any walk continues.
__device__ __forceinline__ void flatten_phase(const FrameArgs& a) {
    constexpr int U = 4;
    const long long n = 2LL * (a.H - 1) * (a.W - 1);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_iter = (n + stride - 1) / stride;   // uniform: whole warps stay together
    const long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int32_t* L = a.labels;
    int32_t* const sizes = a.sizes;
    int32_t* const copy = sizes ? nullptr : a.labels_copy;   // with tri_min the filter writes it
    for (long long it0 = 0; it0 < n_iter; it0 += U) {
        int lab[U], par[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = base + (it0 + u) * stride;
            lab[u] = (it0 + u < n_iter && i < n) ? __ldcg(L + i) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) par[u] = lab[u] >= 0 ? __ldcg(L + lab[u]) : -1;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = base + (it0 + u) * stride;
            int root = -1;
            if (lab[u] >= 0) {
                root = root_from(L, lab[u], par[u]);
                L[i] = root;
            }
            if (copy && it0 + u < n_iter && i < n) copy[i] = root;
            if (sizes) {
                const unsigned peers = __match_any_sync(0xffffffffu, root);
                const int leader = __ffs(peers) - 1;
                if (root >= 0 && (int)(threadIdx.x & 31) == leader) atomicAdd(sizes + root, __popc(peers));
            }
        }
    }
}

// Algorithm 5 keeps a segment only when it has more than tri_min triangles.
__device__ __forceinline__ void filter_phase(const FrameArgs& a) {
    const long long n = 2LL * (a.H - 1) * (a.W - 1);
    int32_t* const labels = a.labels;
    int32_t* const copy = a.labels_copy;
    const int32_t* const sizes = a.sizes;
    const int min_triangles = a.min_triangles;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int l = __ldcg(labels + i);
        const bool drop = l >= 0 && __ldcg(sizes + l) <= min_triangles;   // sizes: other CTAs' atomics
        if (drop) labels[i] = -1;
        if (copy) copy[i] = drop ? -1 : l;
    }
}

__device__ __forceinline__ void phase_mark(const FrameArgs& a, int slot, uint64_t& t_prev) {
    if (a.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t t = global_ns();
        atomicAdd(a.phase_ns + slot, (unsigned long long)(t - t_prev));
        t_prev = t;
    }
}

}  // namespace frame

template <int RL, int RB>
__global__ void __launch_bounds__(kThreads, 2) frame_kernel(const __grid_constant__ FrameArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);   // [kLapMaxStages]: one per staging slot
    float* smem = reinterpret_cast<float*>(smem_raw + 128);
    if (threadIdx.x == 0)
        for (int i = 0; i < kLapMaxStages; ++i) mbar_init(bar + i, 1);
    frame::set_stage_timing(bar, a.phase_ns ? a.phase_ns + kStageSlot : nullptr);
    __syncthreads();
    unsigned par = 0;   // mbarrier parities of the staging slots, one bit each
    uint64_t t_prev = 0;
    if (a.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) t_prev = global_ns();

    // a launch may run part of the path (a.part): the smoothing and tile-local segments, or the
    // segments across tiles; the launch boundary then orders the two
    if (a.part != 2) {
        for (int c = 0; c < a.n_lap; ++c) {
            const LapPhase& ph = a.lap[c];
            const int tiles_lap = ph.tiles;
            const CUtensorMap* map = ph.use_tma ? &a.tm_pts_lap : nullptr;
            // buffers: [box 0 .. box ns-1][D a][D b] (one D buffer for a single-iteration first
            // pass); the box of this CTA's tile k is slot k mod ns, and the TMA loads of its next
            // ns - 1 tiles are in flight while tile k computes
            const int P = align_floats(ph.box.rows * ph.box.cols);
            const int ns = map ? ph.stages : 1;
            float* Da = smem + ns * P;
            float* Db = Da + (ph.dbufs - 1) * P;
            for (int k = 0; k + 1 < ns; ++k) {
                const int t = (int)blockIdx.x + k * (int)gridDim.x;
                if (t < tiles_lap) frame::lap_issue(a, ph, map, t, smem + k * P, bar + k);
            }
            int s = 0;
            for (int t = blockIdx.x; t < tiles_lap; t += gridDim.x) {
                if (map) {
                    const int ahead = t + (ns - 1) * (int)gridDim.x;
                    const int sa = s == 0 ? ns - 1 : s - 1;   // the slot of the previous tile, now free
                    if (ahead < tiles_lap) frame::lap_issue(a, ph, map, ahead, smem + sa * P, bar + sa);
                }
                const frame::LapJob j = frame::lap_job(a, ph, t);
                frame::lap_tile<RL>(j, smem + s * P, Da, Db, map != nullptr, bar + s, (par >> s) & 1u);
                if (map) par ^= 1u << s;
                s = s + 1 == ns ? 0 : s + 1;
            }
            grid_barrier(a.barrier, a.error);
        }
        frame::phase_mark(a, 0, t_prev);
        const int tiles_bil = div_up(a.H - 1, a.bil_th) * div_up(a.W - 1, kTile);
        unsigned par0 = par & 1u;   // the bilateral stages through slot 0
        for (int c = 0; c < a.n_bil; ++c) {
            for (int t = blockIdx.x; t < tiles_bil; t += gridDim.x) frame::bil_tile<RB, true>(a, a.bil[c], t, smem, bar, par0);
            if (a.part == 0 || c + 1 < a.n_bil) grid_barrier(a.barrier, a.error);
        }
        frame::phase_mark(a, 1, t_prev);
    }
    if (a.part == 1) return;
    if (!a.border) {   // else the bilateral tiles joined their borders
        frame::merge_phase(a);
        grid_barrier(a.barrier, a.error);
    }
    frame::phase_mark(a, 2, t_prev);
    frame::flatten_phase(a);
    if (a.min_triangles > 0) {
        grid_barrier(a.barrier, a.error);
        frame::filter_phase(a);
    }
    frame::phase_mark(a, 3, t_prev);
}

namespace frame {

// Frame of work item t: the largest f < n with pre[f] <= t (pre[0] = 0 <= t < pre[n]).
__device__ __forceinline__ int find_frame(const int* pre, int n, int t) {
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(pre + mid) <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Tiles of a batch phase go to the CTAs in runs of kRun consecutive tiles, dealt round-robin.
constexpr int kRun = 4;
__device__ __forceinline__ int next_tile(int t) {
    return (t + 1) % kRun != 0 ? t + 1 : (t / kRun + (int)gridDim.x) * kRun;
}

// Advances f (never backwards) to the frame whose range of pre holds item i.
__device__ __forceinline__ int advance_frame(const long long* pre, int f, long long i) {
    while (__ldg(pre + f + 1) <= i) ++f;
    return f;
}

}  // namespace frame

// Many frames in one persistent launch: each phase runs over the concatenated work of all
// frames (tiles, tile-border twins, triangles), with one grid barrier between phases, so the
// small frames of a batch share the GPU instead of leaving most of it idle.
template <int RL, int RB>
__global__ void __launch_bounds__(kThreads, 2) batch_kernel(const __grid_constant__ BatchArgs b) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);   // [kLapMaxStages]: one per staging slot
    float* smem = reinterpret_cast<float*>(smem_raw + 128);
    if (threadIdx.x == 0)
        for (int i = 0; i < kLapMaxStages; ++i) mbar_init(bar + i, 1);
    frame::set_stage_timing(bar, b.hdr->timing ? b.phase_ns + kStageSlot : nullptr);
    __syncthreads();
    unsigned par = 0;   // mbarrier parities of the staging slots, one bit each
    const int n = b.hdr->n, n_lap = b.hdr->n_lap, n_bil = b.hdr->n_bil;
    const bool any_filter = b.hdr->any_filter != 0;
    unsigned long long* pns = b.hdr->timing ? b.phase_ns : nullptr;
    uint64_t t_prev = 0;
    const bool stamp = pns && blockIdx.x == 0 && threadIdx.x == 0;
    auto mark = [&](int slot) {
        if (stamp) {
            const uint64_t t = global_ns();
            atomicAdd(pns + slot, (unsigned long long)(t - t_prev));
            t_prev = t;
        }
    };
    if (stamp) t_prev = global_ns();

    for (int c = 0; c < n_lap; ++c) {
        const int* pre = b.lap_tiles + c * b.stride;
        const int total = __ldg(pre + n);
        // buffers as in the frame kernel, sized for the largest box of this pass over the frames:
        // [box 0 .. box ns-1][D a][D b]; the box of this CTA's k-th tile is slot k mod ns
        const int P = b.hdr->lap_buf[c];
        const int ns = b.hdr->lap_stages[c];
        float* Da = smem + ns * P;
        float* Db = Da + (b.hdr->lap_dbufs[c] - 1) * P;
        // TMA-issues tile t (of frame f) into a slot when the frame stages by TMA. A CTA meets the
        // frames in increasing order, so it acquires each frame's tensor map once.
        int acquired = -1;
        auto issue = [&](int t, int f, int slot) {
            const FrameArgs& a = b.frames[f];
            if (!a.lap[c].use_tma) return;
            const CUtensorMap* map = &a.tm_pts_lap;
            if (f != acquired) {
                if (threadIdx.x == 0) tensormap_acquire(map);
                acquired = f;
            }
            frame::lap_issue(a, a.lap[c], map, t - __ldg(pre + f), smem + slot * P, bar + slot);
        };
        // runs of kRun consecutive tiles dealt round-robin: neighbouring tiles, whose halos
        // overlap, close together in time, a map acquire per run, and the balance of a
        // round-robin when frames differ in cost
        const int t_begin = (int)blockIdx.x * frame::kRun;
        int f_cur = t_begin < total ? frame::find_frame(pre, n, t_begin) : 0;
        // the furthest tile of the sequence issued so far, and its frame (frames grow along it)
        int t_ahd = t_begin, f_ahd = f_cur;
        if (ns > 1 && t_begin < total) {
            issue(t_begin, f_cur, 0);
            for (int k = 1; k + 1 < ns; ++k) {
                t_ahd = frame::next_tile(t_ahd);
                if (t_ahd >= total) break;
                while (__ldg(pre + f_ahd + 1) <= t_ahd) ++f_ahd;
                issue(t_ahd, f_ahd, k);
            }
        }
        int s = 0;
        for (int t = t_begin; t < total; t = frame::next_tile(t)) {
            while (__ldg(pre + f_cur + 1) <= t) ++f_cur;
            if (ns > 1) {
                t_ahd = frame::next_tile(t_ahd);
                if (t_ahd < total) {
                    while (__ldg(pre + f_ahd + 1) <= t_ahd) ++f_ahd;
                    issue(t_ahd, f_ahd, s == 0 ? ns - 1 : s - 1);   // the previous tile's slot, now free
                }
            } else {
                issue(t, f_cur, 0);
            }
            const FrameArgs& a = b.frames[f_cur];
            const bool tma = a.lap[c].use_tma != 0;
            const frame::LapJob j = frame::lap_job(a, a.lap[c], t - __ldg(pre + f_cur));
            frame::lap_tile<RL>(j, smem + s * P, Da, Db, tma, bar + s, (par >> s) & 1u);
            if (tma) par ^= 1u << s;
            s = s + 1 == ns ? 0 : s + 1;
        }
        grid_barrier(b.barrier, b.error);
    }
    mark(0);
    unsigned par0 = par & 1u;   // the bilateral stages through slot 0
    for (int c = 0; c < n_bil; ++c) {
        const int* pre = b.bil_tiles + c * b.stride;
        const int total = __ldg(pre + n);
        int acquired = -1;   // frames come in increasing order: each frame's maps acquired once
        const int t_begin = (int)blockIdx.x * frame::kRun;
        int f = t_begin < total ? frame::find_frame(pre, n, t_begin) : 0;
        for (int t = t_begin; t < total; t = frame::next_tile(t)) {
            while (__ldg(pre + f + 1) <= t) ++f;
            const FrameArgs& a = b.frames[f];
            if (a.bil[c].use_tma && f != acquired) {
                if (threadIdx.x == 0) {
                    tensormap_acquire(&a.tm_pts_bil);
                    tensormap_acquire(&a.tm_disp_bil);
                }
                acquired = f;
            }
            frame::bil_tile<RB, false>(a, a.bil[c], t - __ldg(pre + f), smem, bar, par0);
        }
        grid_barrier(b.barrier, b.error);
    }
    mark(1);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    {
        const long long total = __ldg(b.merge_items + n);
        const long long n_iter = (total + stride - 1) / stride;   // uniform: whole warps stay together
        int f = 0;
        for (long long it = 0; it < n_iter; ++it) {
            const long long w = base + it * stride;
            int ra = -1, rb = -1;
            bool link = false;
            int32_t* labels = nullptr;
            if (w < total) {
                f = frame::advance_frame(b.merge_items, f, w);
                const FrameArgs& a = b.frames[f];
                labels = a.labels;
                link = frame::merge_pair(a, w - __ldg(b.merge_items + f), ra, rb);
            }
            frame::merge_unite(labels, link, ra, rb, f);
        }
    }
    grid_barrier(b.barrier, b.error);
    mark(2);
    {
        // every grouped triangle takes its root; segment sizes are counted per (frame, root);
        // four triangles per thread in flight at once, as in the single-frame flatten
        constexpr int U = 4;
        const long long total = __ldg(b.tris + n);
        const long long n_iter = (total + stride - 1) / stride;   // uniform: whole warps stay together
        int f = 0;
        for (long long it0 = 0; it0 < n_iter; it0 += U) {
            int lab[U], par[U], fr[U];
            int32_t* lp[U];
            long long li[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long i = base + (it0 + u) * stride;
                lab[u] = -1;
                fr[u] = 0;
                lp[u] = nullptr;
                li[u] = 0;
                if (it0 + u < n_iter && i < total) {
                    f = frame::advance_frame(b.tris, f, i);
                    fr[u] = f;
                    lp[u] = b.frames[f].labels;
                    li[u] = i - __ldg(b.tris + f);
                    lab[u] = __ldcg(lp[u] + li[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) par[u] = lab[u] >= 0 ? __ldcg(lp[u] + lab[u]) : -1;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                int root = -1;
                long long key = -1;
                if (lab[u] >= 0) {
                    root = frame::root_from(lp[u], lab[u], par[u]);
                    lp[u][li[u]] = root;
                    key = ((long long)fr[u] << 32) | (unsigned)root;
                }
                if (any_filter) {
                    const unsigned peers = __match_any_sync(0xffffffffu, key);
                    const int leader = __ffs(peers) - 1;
                    int32_t* sizes = root >= 0 ? b.frames[fr[u]].sizes : nullptr;
                    if (sizes && (int)(threadIdx.x & 31) == leader) atomicAdd(sizes + root, __popc(peers));
                }
            }
        }
    }
    if (any_filter) {
        grid_barrier(b.barrier, b.error);
        // Algorithm 5 keeps a segment only when it has more than tri_min triangles
        const long long total = __ldg(b.tris + n);
        int f = 0;
        for (long long i = base; i < total; i += stride) {
            f = frame::advance_frame(b.tris, f, i);
            const FrameArgs& a = b.frames[f];
            if (!a.sizes) continue;
            const int li = (int)(i - __ldg(b.tris + f));
            const int l = __ldcg(a.labels + li);
            if (l >= 0 && __ldcg(a.sizes + l) <= a.min_triangles) a.labels[li] = -1;
        }
    }
    mark(3);
}

}  // namespace pl3d

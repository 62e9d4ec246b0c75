// lap1.cu -- the Laplacian filter (Eq. 1-2, Section 5.1) at one iteration per pass with a 3 x 3
// window, as a kernel of its own.
//
// A single iteration reads every point once and writes its displacement once (24 bytes per point,
// 36 with the previous pass's displacement), so the pass is bound by HBM and by instruction issue,
// not by the halo trade-off that the fused tile passes of frame_kernels.cuh make. A warp owns a task
// of 64 columns x 24 rows of one frame, each lane a pair of adjacent columns, and walks down its
// rows. Tasks after the first round are handed out by a counter in global memory (a batch mixes
// frames whose ragged tasks differ in size, and a static split leaves a tail of idle warps).
//
// Rows come through a per-warp ring of kRing row slots in shared memory, filled with cp.async:
// one or two 16-byte copies per lane of the row's 800 bytes, from the point left of the chunk to
// the point right of it, when the rows are 16-byte aligned; 4-byte copies per point otherwise.
// So kRing - 4 rows are in flight without holding registers. A lane reads its pair and the points
// on either side of it from the ring (64-bit shared loads, free of bank conflicts at a 24-byte
// stride) into a three-row register window.
//
// A pair shares work that single columns would repeat: the edge between its two points (E of the
// left one, W of the right one), the vertical edges (S of a row is N of the next), and the two
// diagonals inside the pair (SE of the left point and SW of the right one become NW and NE of the
// next row's pair). Only the weight of a shared diagonal is kept; its difference is formed again.
//
// Every point is the same arithmetic as in lap_iteration (frame_kernels.cuh): its window in
// row-major order (NW, N, NE, W, E, SW, S, SE), a shared edge entering with its difference negated
// (w_ij = w_ji, opposite differences), the same rounding intrinsics. Passes of this kernel and fused
// tile passes therefore give the same bits, and a batch the same bits as single frames.
//
// Invalid points (any coordinate non-finite or beyond kMaxCoord, and points outside the image)
// become the finite sentinel kInvalidCoord with zero displacement, whose weight underflows to 0.
#include "frame_kernels.cuh"

namespace pl3d {
namespace frame {
namespace {

constexpr int kWarps = kLap1Threads / 32;
constexpr int kBlock = 3;      // rows per unrolled block: the register window's period
// Row slots of a warp's ring: rows i + 3 .. i + kRing - 2 in flight at row i.
template <bool WITH_D>
struct L1Ring {
    static constexpr int n = WITH_D ? 8 : 8;
};
// A slot: float 0 pad, floats 1-3 the point left of the chunk, floats 4 .. 195 the chunk's 64
// points, floats 196-198 the point right of it, float 199 pad; kSlot / 4 pieces of 16 bytes.
constexpr int kSlot = 200;
constexpr int kSlotPts = 4;
constexpr int kPieces = kSlot / 4;
static_assert(kLap1Cols == 64 && kLap1Rows % kBlock == 0, "warp tasks: 64 columns, whole blocks of rows");
static_assert(kSlotPts + 3 * kLap1Cols + 3 <= kSlot && kPieces <= 64, "slot layout");

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One row of the window: the point left of the lane's pair, the pair (a, b), the point right of it.
struct L1Row {
    LapPt l, a, b, r;
};

struct L1Geom {
    int H, W, c0, lane;
    bool vec;     // 16-byte copies: rows 16-byte aligned (W % 4 == 0, aligned arrays)
    // vec: the lane's two pieces (lane, lane + 32): float offsets in the row, and whether each
    // lies inside the row (with W % 4 == 0 a piece lies wholly inside or wholly outside)
    int f0, f1;
    bool in0, in1;
};

__device__ __forceinline__ void l1_geom_pieces(L1Geom& g) {
    g.f0 = 3 * g.c0 - kSlotPts + 4 * g.lane;
    g.f1 = g.f0 + 4 * 32;
    g.in0 = g.f0 >= 0 && g.f0 + 4 <= 3 * g.W;
    g.in1 = g.lane + 32 < kPieces && g.f1 + 4 <= 3 * g.W;
}

// The edge from a point to the one below it: difference (below - point) and its weight.
struct L1Edge {
    float ex, ey, ez, w;
};

// Copies row `row` of the AoS array A (points or displacements) into a ring slot: the warp's 64
// points and the one point on each side; points outside the image read as `fill`.
__device__ __forceinline__ void l1_fill(float* slot, const float* A, const L1Geom& g, int row, float fill) {
    const int lane = g.lane;
    const float4 f4 = make_float4(fill, fill, fill, fill);
    if ((unsigned)row >= (unsigned)g.H) {
        *reinterpret_cast<float4*>(slot + 4 * lane) = f4;
        if (lane + 32 < kPieces) *reinterpret_cast<float4*>(slot + 4 * (lane + 32)) = f4;
        return;
    }
    const float* rowp = A + (long long)row * (3 * g.W);   // 3 H W < 2^31 floats (pl3d_validate)
    if (g.vec) {
        // the pieces of the floats 3 c0 - 4 .. 3 c0 + 195 of the row; one outside it reads as fill
        if (g.in0) cp_async16(slot + 4 * lane, rowp + g.f0);
        else *reinterpret_cast<float4*>(slot + 4 * lane) = f4;
        if (lane + 32 < kPieces) {
            if (g.in1) cp_async16(slot + 4 * (lane + 32), rowp + g.f1);
            else *reinterpret_cast<float4*>(slot + 4 * (lane + 32)) = f4;
        }
        return;
    }
    // point by point: the lane's pair, and the point on each side for lanes 0 and 31
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int c = g.c0 + 2 * lane + k;
        float* d = slot + kSlotPts + 3 * (2 * lane + k);
        if (c < g.W) {
            cp_async4(d, rowp + 3 * c);
            cp_async4(d + 1, rowp + 3 * c + 1);
            cp_async4(d + 2, rowp + 3 * c + 2);
        } else {
            d[0] = d[1] = d[2] = fill;
        }
    }
    if (lane == 0 || lane == 31) {
        const int c = lane == 0 ? g.c0 - 1 : g.c0 + kLap1Cols;
        float* d = lane == 0 ? slot + 1 : slot + kSlotPts + 3 * kLap1Cols;
        if (c >= 0 && c < g.W) {
            cp_async4(d, rowp + 3 * c);
            cp_async4(d + 1, rowp + 3 * c + 1);
            cp_async4(d + 2, rowp + 3 * c + 2);
        } else {
            d[0] = d[1] = d[2] = fill;
        }
    }
}

// Invalid -> the sentinel with zero displacement.
template <bool WITH_D>
__device__ __forceinline__ LapPt l1_point(float x, float y, float z, float dx, float dy, float dz) {
    LapPt q;
    const bool ok = point_valid(x, y, z);
    q.x = ok ? x : kInvalidCoord;
    q.y = ok ? y : kInvalidCoord;
    q.z = ok ? z : kInvalidCoord;
    q.dx = (WITH_D && ok) ? dx : 0.f;
    q.dy = (WITH_D && ok) ? dy : 0.f;
    q.dz = (WITH_D && ok) ? dz : 0.f;
    return q;
}

// The 12 floats of a lane's window row: the left point at slot float 1 + 6 lane, the pair at
// 4 + 6 lane, the right point at 10 + 6 lane (64-bit loads at the even offsets).
struct L1Floats {
    float v[12];
};

__device__ __forceinline__ void l1_read(const float* s, int lane, L1Floats& f) {
    const int o = 6 * lane;
    f.v[0] = s[o + 1];
    const float2 p0 = *reinterpret_cast<const float2*>(s + o + 2);
    const float2 p1 = *reinterpret_cast<const float2*>(s + o + 4);
    const float2 p2 = *reinterpret_cast<const float2*>(s + o + 6);
    const float2 p3 = *reinterpret_cast<const float2*>(s + o + 8);
    const float2 p4 = *reinterpret_cast<const float2*>(s + o + 10);
    f.v[1] = p0.x, f.v[2] = p0.y, f.v[3] = p1.x, f.v[4] = p1.y, f.v[5] = p2.x, f.v[6] = p2.y;
    f.v[7] = p3.x, f.v[8] = p3.y, f.v[9] = p4.x, f.v[10] = p4.y;
    f.v[11] = s[o + 12];
}

template <bool WITH_D>
__device__ __forceinline__ void l1_take(const float* sp, const float* sd, int lane, L1Row& w) {
    L1Floats p, d;
    l1_read(sp, lane, p);
    if (WITH_D) {
        l1_read(sd, lane, d);
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) d.v[k] = 0.f;
    }
    w.l = l1_point<WITH_D>(p.v[0], p.v[1], p.v[2], d.v[0], d.v[1], d.v[2]);
    w.a = l1_point<WITH_D>(p.v[3], p.v[4], p.v[5], d.v[3], d.v[4], d.v[5]);
    w.b = l1_point<WITH_D>(p.v[6], p.v[7], p.v[8], d.v[6], d.v[7], d.v[8]);
    w.r = l1_point<WITH_D>(p.v[9], p.v[10], p.v[11], d.v[9], d.v[10], d.v[11]);
}

// Frame f of warp task t: the largest f < n with pre[f] <= t (pre[0] = 0 <= t < pre[n]). The
// lanes probe 32 positions at once.
__device__ __forceinline__ int l1_find_frame(const int* pre, int n, int t, int lane) {
    int lo = 0, hi = n;   // pre[lo] <= t < pre[hi]
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int pos = lo + lane * step;
        const bool le = pos < hi && __ldg(pre + pos) <= t;
        const unsigned m = __ballot_sync(0xffffffffu, le);   // lanes 0 .. k (lane 0: pos = lo)
        const int k = 31 - __clz((int)m);
        lo += k * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Sums of one point's Eq. 1 terms.
struct L1Sum {
    float sx, sy, sz, ws;
};

// A neighbour term with a fresh difference q - p and its weight.
template <bool WITH_D>
__device__ __forceinline__ void l1_add(L1Sum& s, const LapPt& p, const LapPt& q) {
    float ex, ey, ez;
    lap_diff<WITH_D>(p, q, ex, ey, ez);
    lap_accumulate(s.sx, s.sy, s.sz, s.ws, lap_weight(ex, ey, ez), ex, ey, ez);
}

// A neighbour term with a fresh difference q - p and a known weight (of the same pair of points).
template <bool WITH_D>
__device__ __forceinline__ void l1_add_w(L1Sum& s, const LapPt& p, const LapPt& q, float w) {
    float ex, ey, ez;
    lap_diff<WITH_D>(p, q, ex, ey, ez);
    lap_accumulate(s.sx, s.sy, s.sz, s.ws, w, ex, ey, ez);
}

// A neighbour term whose difference is the negation of a known edge's (the edge from q to p).
__device__ __forceinline__ void l1_add_neg(L1Sum& s, const L1Edge& e) {
    lap_accumulate(s.sx, s.sy, s.sz, s.ws, e.w, -e.ex, -e.ey, -e.ez);
}

// A neighbour term that also keeps its edge (difference q - p and weight).
template <bool WITH_D>
__device__ __forceinline__ void l1_add_keep(L1Sum& s, const LapPt& p, const LapPt& q, L1Edge& e) {
    lap_diff<WITH_D>(p, q, e.ex, e.ey, e.ez);
    e.w = lap_weight(e.ex, e.ey, e.ez);
    lap_accumulate(s.sx, s.sy, s.sz, s.ws, e.w, e.ex, e.ey, e.ez);
}

// Eq. 1 for one point: its new displacement, or the kept one.
__device__ __forceinline__ void l1_out(const LapPt& p, const L1Sum& s, bool pin, float lambda, float& ox, float& oy,
                                       float& oz) {
    const bool keep = pin || p.x == kInvalidCoord || !(s.ws > 0.f);
    const float k = lap_scale(keep, lambda, s.ws);
    ox = fmaf(k, s.sx, p.dx);
    oy = fmaf(k, s.sy, p.dy);
    oz = fmaf(k, s.sz, p.dz);
}

__device__ __forceinline__ void l1_export(float* e, const LapPt& p, float ox, float oy, float oz) {
    const bool valid = p.x != kInvalidCoord;
    e[0] = valid ? __fadd_rn(p.x, ox) : NAN;
    e[1] = valid ? __fadd_rn(p.y, oy) : NAN;
    e[2] = valid ? __fadd_rn(p.z, oz) : NAN;
}

// One warp task: columns cb * 64 + 2 lane and + 1, rows rb * kLap1Rows .. + kLap1Rows - 1 of frame
// fr. `ring` (and `dring` with WITH_D) hold kRing slots of this warp.
template <bool WITH_D>
__device__ __forceinline__ void l1_task(const Lap1Frame& fr, int task, int lane, float* ring, float* dring) {
    constexpr int kRing = L1Ring<WITH_D>::n;
    const int H = fr.H, W = fr.W;
    const int ncb = div_up(W, kLap1Cols);
    const int rb = task / ncb, cb = task - rb * ncb;
    const int r0 = rb * kLap1Rows;
    L1Geom g;
    g.H = H;
    g.W = W;
    g.c0 = cb * kLap1Cols;
    g.lane = lane;
    g.vec = (W & 3) == 0 && ((uintptr_t)fr.points & 15u) == 0 && (!WITH_D || ((uintptr_t)fr.d_in & 15u) == 0);
    l1_geom_pieces(g);
    const int ca = g.c0 + 2 * lane;   // the pair's columns: ca, ca + 1
    const bool out_a = ca < W, out_b = ca + 1 < W;
    const bool pin_a = ca < 1 || ca >= W - 1, pin_b = ca + 1 >= W - 1;
    const float lambda = fr.lambda;
    float* const d_out = fr.d_out;
    float* const exp_pts = fr.export_points;
    if (fr.iters == 0) {
        // no smoothing: the displacement stays zero (warp-uniform; only a first pass has no iteration)
        for (int r = r0; r < min(H, r0 + kLap1Rows); ++r) {
            const size_t gi = 3 * ((size_t)r * W + ca);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!(k == 0 ? out_a : out_b)) continue;
                const size_t o = gi + 3 * k;
                d_out[o] = d_out[o + 1] = d_out[o + 2] = 0.f;
                if (exp_pts) {
                    const float x = __ldg(fr.points + o), y = __ldg(fr.points + o + 1), z = __ldg(fr.points + o + 2);
                    l1_export(exp_pts + o, l1_point<false>(x, y, z, 0.f, 0.f, 0.f), 0.f, 0.f, 0.f);
                }
            }
        }
        return;
    }
    // the pair's six floats start 8-byte aligned in every row when W is even
    const bool st64 = (W & 1) == 0 && ((uintptr_t)d_out & 7u) == 0;
    // rows r0 - 1 .. r0 + kLap1Rows are needed (row H, the one below the image, read as invalid);
    // ring index i holds row r0 - 1 + i in slot i % kRing
    const int last_index = min(kLap1Rows + 1, H - r0 + 1);
    auto fill = [&](int i) {
        if (i <= last_index) {
            l1_fill(ring + (i % kRing) * kSlot, fr.points, g, r0 - 1 + i, NAN);
            if (WITH_D) l1_fill(dring + (i % kRing) * kSlot, fr.d_in, g, r0 - 1 + i, 0.f);
        }
        cp_async_commit();   // one group per index, empty or not: the wait counts stay constant
    };
    auto take = [&](int i, L1Row& w) {
        const int o = (i % kRing) * kSlot;
        l1_take<WITH_D>(ring + o, WITH_D ? dring + o : ring + o, lane, w);
    };

    L1Row win[3];
    // prologue: indices 0 .. kRing - 2 in flight; rows r0 - 1, r0, r0 + 1 into window slots 2, 0, 1
    for (int i = 0; i + 1 < kRing; ++i) fill(i);
    cp_async_wait<kRing - 4>();
    __syncwarp();
    take(0, win[2]);
    take(1, win[0]);
    take(2, win[1]);
    // edges carried from row r - 1 to row r: the verticals of a and b, and the weights of the
    // diagonals inside the pair (a above to b below, b above to a below)
    L1Edge na, nb;
    float w_se, w_sw;
    {
        const L1Row& up = win[2];
        const L1Row& mid = win[0];
        lap_diff<WITH_D>(up.a, mid.a, na.ex, na.ey, na.ez);
        na.w = lap_weight(na.ex, na.ey, na.ez);
        lap_diff<WITH_D>(up.b, mid.b, nb.ex, nb.ey, nb.ez);
        nb.w = lap_weight(nb.ex, nb.ey, nb.ez);
        float ex, ey, ez;
        lap_diff<WITH_D>(up.a, mid.b, ex, ey, ez);
        w_se = lap_weight(ex, ey, ez);
        lap_diff<WITH_D>(up.b, mid.a, ex, ey, ez);
        w_sw = lap_weight(ex, ey, ez);
    }

    for (int bk = 0; bk < kLap1Rows; bk += kBlock) {
        if (r0 + bk >= H) break;   // warp-uniform
#pragma unroll
        for (int j = 0; j < kBlock; ++j) {
            const int r = r0 + bk + j;
            const int i = bk + j + 1;   // ring index of row r
            L1Row& up = win[(j + 2) % 3];
            L1Row& mid = win[j % 3];
            L1Row& dn = win[(j + 1) % 3];
            fill(i + kRing - 2);   // into the slot of index i - 2, read before the last __syncwarp

            const LapPt& pa = mid.a;
            const LapPt& pb = mid.b;
            L1Sum A = {0.f, 0.f, 0.f, 0.f}, B = {0.f, 0.f, 0.f, 0.f};
            // a: NW, N (carried), NE (weight carried), W
            l1_add<WITH_D>(A, pa, up.l);
            l1_add_neg(A, na);
            l1_add_w<WITH_D>(A, pa, up.b, w_sw);
            l1_add<WITH_D>(A, pa, mid.l);
            // b: NW (weight carried), N (carried), NE
            l1_add_w<WITH_D>(B, pb, up.a, w_se);
            l1_add_neg(B, nb);
            l1_add<WITH_D>(B, pb, up.r);
            // the edge inside the pair: E of a, W of b
            L1Edge ab;
            l1_add_keep<WITH_D>(A, pa, pb, ab);
            l1_add_neg(B, ab);
            // a: SW, S (kept for the next row), SE (weight kept)
            l1_add<WITH_D>(A, pa, dn.l);
            l1_add_keep<WITH_D>(A, pa, dn.a, na);
            L1Edge dg;
            l1_add_keep<WITH_D>(A, pa, dn.b, dg);
            w_se = dg.w;
            // b: E, SW (weight kept), S (kept), SE
            l1_add<WITH_D>(B, pb, mid.r);
            l1_add_keep<WITH_D>(B, pb, dn.a, dg);
            w_sw = dg.w;
            l1_add_keep<WITH_D>(B, pb, dn.b, nb);
            l1_add<WITH_D>(B, pb, dn.r);

            const bool row_pin = r < 1 || r >= H - 1;
            float ax, ay, az, bx, by, bz;
            l1_out(pa, A, pin_a || row_pin, lambda, ax, ay, az);
            l1_out(pb, B, pin_b || row_pin, lambda, bx, by, bz);
            if (r < H) {   // warp-uniform
                const long long gi = (long long)r * (3 * W) + 3 * ca;
                if (st64 && out_b) {
                    float2* o = reinterpret_cast<float2*>(d_out + gi);
                    o[0] = make_float2(ax, ay);
                    o[1] = make_float2(az, bx);
                    o[2] = make_float2(by, bz);
                } else {
                    if (out_a) {
                        d_out[gi] = ax;
                        d_out[gi + 1] = ay;
                        d_out[gi + 2] = az;
                    }
                    if (out_b) {
                        d_out[gi + 3] = bx;
                        d_out[gi + 4] = by;
                        d_out[gi + 5] = bz;
                    }
                }
                if (exp_pts) {
                    if (out_a) l1_export(exp_pts + gi, pa, ax, ay, az);
                    if (out_b) l1_export(exp_pts + gi + 3, pb, bx, by, bz);
                }
            }
            // row r + 2 (index i + 2) takes the window slot of row r - 1
            cp_async_wait<kRing - 4>();
            __syncwarp();
            take(i + 2, up);
        }
    }
    // nothing of this task may still be landing in the ring when the next task fills it
    cp_async_wait<0>();
    __syncwarp();
}

}  // namespace
}  // namespace frame

size_t lap1_smem_bytes(bool with_d) {
    const int slots = with_d ? 2 * frame::L1Ring<true>::n : frame::L1Ring<false>::n;
    return (size_t)slots * frame::kWarps * frame::kSlot * sizeof(float);
}

// Dynamic shared memory: kWarps rings of points, then (WITH_D) kWarps rings of displacements.
// Four-warp CTAs, five per SM (96 registers, no spills; four with the displacement window at 128):
// 20 warps per SM measured faster than 24 at 80 registers with spills, and than 16 at 128.
template <bool WITH_D>
__global__ void __launch_bounds__(kLap1Threads, WITH_D ? kLap1CtasD : kLap1Ctas) lap1_kernel(const __grid_constant__ Lap1Args a) {
    extern __shared__ __align__(16) float l1_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarpFloats = frame::L1Ring<WITH_D>::n * frame::kSlot;
    float* const ring = l1_smem + warp * kWarpFloats;
    float* const dring = WITH_D ? l1_smem + (frame::kWarps + warp) * kWarpFloats : ring;
    bool timed = false;
    if (a.stamp) timed = a.hdr ? __ldg(&a.hdr->timing) != 0 : true;
    if (timed && threadIdx.x == 0) atomicMax(a.stamp, ~(unsigned long long)global_ns());
    const int n = a.hdr ? __ldg(&a.hdr->n) : 1;
    const int tasks = a.hdr ? __ldg(a.task_pre + n) : lap1_tasks(a.one.H, a.one.W);
    // The first round of tasks goes one per warp by index; after it, a warp takes the next task
    // from the counter, asked for when it starts a task, so that the warps end within about one
    // task of each other however the frames' ragged tasks fall.
    const int warps = gridDim.x * frame::kWarps;
    int t = blockIdx.x * frame::kWarps + warp;
    while (t < tasks) {
        unsigned next = 0;
        if (lane == 0) next = atomicAdd(a.sched, 1u);
        if (a.hdr) {
            const int f = frame::l1_find_frame(a.task_pre, n, t, lane);
            const FrameArgs* fa = a.frames + f;
            const LapPhase* ph = &fa->lap[a.pass];
            Lap1Frame fr;
            fr.points = reinterpret_cast<const float*>(__ldg(reinterpret_cast<const unsigned long long*>(&fa->points)));
            fr.d_in = reinterpret_cast<const float*>(__ldg(reinterpret_cast<const unsigned long long*>(&ph->d_in)));
            fr.d_out = reinterpret_cast<float*>(__ldg(reinterpret_cast<const unsigned long long*>(&ph->d_out)));
            fr.export_points =
                reinterpret_cast<float*>(__ldg(reinterpret_cast<const unsigned long long*>(&ph->export_points)));
            fr.H = __ldg(&fa->H);
            fr.W = __ldg(&fa->W);
            fr.iters = __ldg(&ph->iters);
            fr.lambda = __ldg(&fa->lambda);
            frame::l1_task<WITH_D>(fr, t - __ldg(a.task_pre + f), lane, ring, dring);
        } else {
            frame::l1_task<WITH_D>(a.one, t, lane, ring, dring);
        }
        t = warps + (int)__shfl_sync(0xffffffffu, next, 0);
    }
    // every warp of every CTA has taken its last index before the last CTA puts the counter back
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.sched + 1, 1u) + 1 == gridDim.x) {
            atomicExch(a.sched, 0u);
            atomicExch(a.sched + 1, 0u);
        }
    }
    if (timed) {
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicMax(a.stamp + 1, (unsigned long long)global_ns());
            __threadfence();
            if (atomicAdd(a.stamp + 2, 1ull) + 1 == gridDim.x) {
                __threadfence();
                const unsigned long long t0 = ~atomicAdd(a.stamp, 0ull), t1 = atomicAdd(a.stamp + 1, 0ull);
                atomicAdd(a.phase_ns, t1 - t0);
                a.stamp[0] = 0;
                a.stamp[1] = 0;
                a.stamp[2] = 0;
            }
        }
    }
}

template __global__ void lap1_kernel<false>(const __grid_constant__ Lap1Args a);
template __global__ void lap1_kernel<true>(const __grid_constant__ Lap1Args a);

const void* lap1_kernel_for(bool with_d) {
    return with_d ? reinterpret_cast<const void*>(&lap1_kernel<true>) : reinterpret_cast<const void*>(&lap1_kernel<false>);
}

}  // namespace pl3d

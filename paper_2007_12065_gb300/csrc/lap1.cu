// lap1.cu -- the Laplacian filter (Eq. 1-2, Section 5.1) at one iteration per pass with a 3 x 3
// window, as a kernel of its own.
//
// A single iteration reads every point once and writes its displacement once (24 bytes per point,
// 36 with the previous pass's displacement), so the pass is bound by HBM, by instruction issue and
// by how many loads are in flight, not by the halo trade-off that the fused tile passes of
// frame_kernels.cuh make. A warp owns a task of 32 columns x 24 rows of one frame, each lane one
// column, and walks down its rows. The rows come through a per-warp ring of kRing row slots in
// shared memory, filled with cp.async (16-byte copies of the warp's 384-byte row chunk when the
// rows are 16-byte aligned, 4-byte copies per point otherwise; lanes 0 and 31 also copy the point
// just outside the chunk), so that kRing - 4 rows are in flight without holding registers. A lane
// reads its point and its left and right neighbours of a row from the ring into a three-row
// register window, where the point is computed.
//
// Every point is the same arithmetic as in lap_iteration (frame_kernels.cuh): its window in
// row-major order (NW, N, NE, W, E, SW, S, SE), the edge to the row below shared with that row's
// point (w_ij = w_ji, opposite differences), the same rounding intrinsics. Passes of this kernel
// and fused tile passes therefore give the same bits, and a batch the same bits as single frames.
//
// Invalid points (any coordinate non-finite or beyond kMaxCoord, and points outside the image)
// become the finite sentinel kInvalidCoord with zero displacement, whose weight underflows to 0.
#include "frame_kernels.cuh"

namespace pl3d {
namespace frame {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = kThreads / 32;
constexpr int kBlock = 3;      // rows per unrolled block: the register window's period
constexpr int kRing = 8;       // row slots of a warp's ring: rows i + 3 .. i + 6 in flight at row i
constexpr int kSlot = 104;     // floats per slot: pad, left point, 32 points (at float 4), right point, pad
constexpr int kSlotPts = 4;    // float offset of the chunk's first point (16-byte aligned)
static_assert(kLap1Rows % kBlock == 0, "warp tasks are whole blocks of rows");
static_assert(kSlot % 4 == 0 && kSlotPts + 96 + 3 <= kSlot, "slot layout");

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

// One row of the window: the lane's point and its left and right neighbours.
struct L1Row {
    LapPt l, c, r;
};

struct L1Geom {
    int H, W, c0, lane;
    int nvalid;   // points of the image in this warp's 32 columns
    bool vec;     // 16-byte copies: rows 16-byte aligned (W % 4 == 0, aligned arrays)
};

// Copies row `row` of the AoS array A (points or displacements) into a ring slot: the warp's 32
// points and the one point on each side; points outside the image read as `fill`.
__device__ __forceinline__ void l1_fill(float* slot, const float* A, const L1Geom& g, int row, float fill) {
    const int lane = g.lane;
    if (row < 0 || row >= g.H) {
        slot[kSlotPts + 3 * lane] = fill;
        slot[kSlotPts + 3 * lane + 1] = fill;
        slot[kSlotPts + 3 * lane + 2] = fill;
        if (lane == 0) slot[1] = slot[2] = slot[3] = fill;
        if (lane == 31) slot[kSlotPts + 96] = slot[kSlotPts + 97] = slot[kSlotPts + 98] = fill;
        return;
    }
    const float* src = A + 3 * ((size_t)row * g.W + g.c0);
    if (g.vec) {
        // 3 nvalid floats, a multiple of 4 when W is: whole 16-byte pieces of the valid points
        if (lane < 24 && 4 * lane < 3 * g.nvalid) cp_async16(slot + kSlotPts + 4 * lane, src + 4 * lane);
    } else if (lane < g.nvalid) {
        cp_async4(slot + kSlotPts + 3 * lane, src + 3 * lane);
        cp_async4(slot + kSlotPts + 3 * lane + 1, src + 3 * lane + 1);
        cp_async4(slot + kSlotPts + 3 * lane + 2, src + 3 * lane + 2);
    }
    if (lane >= g.nvalid) {
        slot[kSlotPts + 3 * lane] = fill;
        slot[kSlotPts + 3 * lane + 1] = fill;
        slot[kSlotPts + 3 * lane + 2] = fill;
    }
    if (lane == 0) {
        if (g.c0 > 0) {
            cp_async4(slot + 1, src - 3);
            cp_async4(slot + 2, src - 2);
            cp_async4(slot + 3, src - 1);
        } else {
            slot[1] = slot[2] = slot[3] = fill;
        }
    }
    if (lane == 31) {
        if (g.nvalid == 32 && g.c0 + 32 < g.W) {
            cp_async4(slot + kSlotPts + 96, src + 96);
            cp_async4(slot + kSlotPts + 97, src + 97);
            cp_async4(slot + kSlotPts + 98, src + 98);
        } else {
            slot[kSlotPts + 96] = slot[kSlotPts + 97] = slot[kSlotPts + 98] = fill;
        }
    }
}

// Invalid -> the sentinel with zero displacement.
template <bool WITH_D>
__device__ __forceinline__ LapPt l1_point(const float* p, const float* d) {
    LapPt q;
    const float x = p[0], y = p[1], z = p[2];
    const bool ok = point_valid(x, y, z);
    q.x = ok ? x : kInvalidCoord;
    q.y = ok ? y : kInvalidCoord;
    q.z = ok ? z : kInvalidCoord;
    q.dx = (WITH_D && ok) ? d[0] : 0.f;
    q.dy = (WITH_D && ok) ? d[1] : 0.f;
    q.dz = (WITH_D && ok) ? d[2] : 0.f;
    return q;
}

// The lane's left point, own point and right point of a ring slot into a window row.
template <bool WITH_D>
__device__ __forceinline__ void l1_take(const float* sp, const float* sd, int lane, L1Row& w) {
    const int o = kSlotPts + 3 * lane;
    w.l = l1_point<WITH_D>(sp + o - 3, sd + o - 3);
    w.c = l1_point<WITH_D>(sp + o, sd + o);
    w.r = l1_point<WITH_D>(sp + o + 3, sd + o + 3);
}

// The shared edge to the row below: difference (below - centre) and its weight.
struct L1Edge {
    float ex, ey, ez, w;
};

// Frame f of warp task t: the largest f < n with pre[f] <= t (pre[0] = 0 <= t < pre[n]). The
// lanes probe 32 positions at once.
__device__ __forceinline__ int l1_find_frame(const int* pre, int n, int t, int lane) {
    int lo = 0, hi = n;   // pre[lo] <= t < pre[hi]
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int pos = lo + lane * step;
        const bool le = pos < hi && __ldg(pre + pos) <= t;
        const unsigned m = __ballot_sync(kFull, le);   // lanes 0 .. k (lane 0: pos = lo)
        const int k = 31 - __clz((int)m);
        lo += k * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// One warp task: columns cb * 32 + lane, rows rb * kLap1Rows .. + kLap1Rows - 1 of frame fr. `ring`
// (and `dring` with WITH_D) hold kRing slots; `stage` one output row.
template <bool WITH_D>
__device__ __forceinline__ void l1_task(const Lap1Frame& fr, int task, int lane, float* ring, float* dring,
                                        float* stage) {
    const int H = fr.H, W = fr.W;
    const int ncb = div_up(W, kLap1Cols);
    const int rb = task / ncb, cb = task - rb * ncb;
    const int r0 = rb * kLap1Rows;
    L1Geom g;
    g.H = H;
    g.W = W;
    g.c0 = cb * kLap1Cols;
    g.lane = lane;
    g.nvalid = min(32, W - g.c0);
    g.vec = (W & 3) == 0 && ((uintptr_t)fr.points & 15u) == 0 && (!WITH_D || ((uintptr_t)fr.d_in & 15u) == 0);
    const int c = g.c0 + lane;
    const bool col_out = c < W;
    const float lambda = fr.lambda;
    const bool zero = fr.iters == 0;
    float* const d_out = fr.d_out;
    float* const exp_pts = fr.export_points;
    // rows go out as float4 through the staging row when they are 16-byte aligned
    const bool vec_out = (W & 3) == 0 && ((uintptr_t)d_out & 15u) == 0;
    const bool colpin = c < 1 || c >= W - 1;
    // rows r0 - 1 .. r0 + kLap1Rows are needed (row H, the one below the image, read as invalid);
    // ring index i holds row r0 - 1 + i in slot i % kRing
    const int last_index = min(kLap1Rows + 1, H - r0 + 1);
    auto fill = [&](int i) {
        if (i <= last_index) {
            float* sl = ring + (i % kRing) * kSlot;
            l1_fill(sl, fr.points, g, r0 - 1 + i, NAN);
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
    L1Edge es;   // edge from row r - 1 down to row r of this column
    lap_diff<WITH_D>(win[2].c, win[0].c, es.ex, es.ey, es.ez);
    es.w = lap_weight(es.ex, es.ey, es.ez);

    for (int b = 0; b < kLap1Rows; b += kBlock) {
        if (r0 + b >= H) break;   // warp-uniform
#pragma unroll
        for (int j = 0; j < kBlock; ++j) {
            const int r = r0 + b + j;
            const int i = b + j + 1;   // ring index of row r
            L1Row& up = win[(j + 2) % 3];
            L1Row& mid = win[j % 3];
            L1Row& dn = win[(j + 1) % 3];
            fill(i + kRing - 2);   // into the slot of index i - 2, read before the last __syncwarp

            LapAcc A;
            A.c = mid.c;
            A.sx = A.sy = A.sz = A.ws = 0.f;
            lap_add<WITH_D>(A, up.l);                                                   // NW
            lap_accumulate(A.sx, A.sy, A.sz, A.ws, es.w, -es.ex, -es.ey, -es.ez);      // N (shared)
            lap_add<WITH_D>(A, up.r);                                                   // NE
            lap_add<WITH_D>(A, mid.l);                                                  // W
            lap_add<WITH_D>(A, mid.r);                                                  // E
            lap_add<WITH_D>(A, dn.l);                                                   // SW
            lap_diff<WITH_D>(A.c, dn.c, es.ex, es.ey, es.ez);                           // S (kept)
            es.w = lap_weight(es.ex, es.ey, es.ez);
            lap_accumulate(A.sx, A.sy, A.sz, A.ws, es.w, es.ex, es.ey, es.ez);
            lap_add<WITH_D>(A, dn.r);                                                   // SE

            const bool keep = colpin || r < 1 || r >= H - 1 || A.c.x == kInvalidCoord || !(A.ws > 0.f);
            const float s = lap_scale(keep, lambda, A.ws);
            float ox = fmaf(s, A.sx, A.c.dx), oy = fmaf(s, A.sy, A.c.dy), oz = fmaf(s, A.sz, A.c.dz);
            if (zero) ox = oy = oz = 0.f;
            if (r < H) {   // warp-uniform
                const size_t gi = 3 * ((size_t)r * W + c);
                if (vec_out) {
                    stage[3 * lane] = ox;
                    stage[3 * lane + 1] = oy;
                    stage[3 * lane + 2] = oz;
                    __syncwarp();
                    if (lane < 24 && 4 * lane < 3 * g.nvalid)
                        *reinterpret_cast<float4*>(d_out + 3 * ((size_t)r * W + g.c0) + 4 * lane) =
                            reinterpret_cast<const float4*>(stage)[lane];
                    __syncwarp();
                } else if (col_out) {
                    d_out[gi] = ox;
                    d_out[gi + 1] = oy;
                    d_out[gi + 2] = oz;
                }
                if (exp_pts && col_out) {
                    const bool valid = A.c.x != kInvalidCoord;
                    exp_pts[gi] = valid ? __fadd_rn(A.c.x, ox) : NAN;
                    exp_pts[gi + 1] = valid ? __fadd_rn(A.c.y, oy) : NAN;
                    exp_pts[gi + 2] = valid ? __fadd_rn(A.c.z, oz) : NAN;
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

template <bool WITH_D>
__global__ void __launch_bounds__(kThreads, WITH_D ? 2 : 4) lap1_kernel(const __grid_constant__ Lap1Args a) {
    __shared__ __align__(16) float stage[kThreads / 32][3 * 32];
    __shared__ __align__(16) float ring[kThreads / 32][frame::kRing * frame::kSlot];
    __shared__ __align__(16) float dring[WITH_D ? kThreads / 32 : 1][WITH_D ? frame::kRing * frame::kSlot : 4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool timed = false;
    if (a.stamp) timed = a.hdr ? __ldg(&a.hdr->timing) != 0 : true;
    if (timed && threadIdx.x == 0) atomicMax(a.stamp, ~(unsigned long long)global_ns());
    const int n = a.hdr ? __ldg(&a.hdr->n) : 1;
    const int tasks = a.hdr ? __ldg(a.task_pre + n) : lap1_tasks(a.one.H, a.one.W);
    for (int t = blockIdx.x * frame::kWarps + warp; t < tasks; t += gridDim.x * frame::kWarps) {
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
            frame::l1_task<WITH_D>(fr, t - __ldg(a.task_pre + f), lane, ring[warp], dring[WITH_D ? warp : 0],
                                   stage[warp]);
        } else {
            frame::l1_task<WITH_D>(a.one, t, lane, ring[warp], dring[WITH_D ? warp : 0], stage[warp]);
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

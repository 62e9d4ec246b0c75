// lap_smooth.cu -- Laplacian vertex smoothing on the implicit image grid (Eq. 1-2, Section 5.1).
//
// Update of a valid interior point v with the valid points v_j of its k x k window
// (itself and points at distance 0 excluded):
//     w_j = 1 / |v_j - v|                                 (Eq. 2)
//     v'  = v + lambda * sum_j w_j (v_j - v) / sum_j w_j  (Eq. 1, umbrella form)
// Invalid points stay invalid, points with no usable neighbour stay put, and the ring of width
// k/2 at the image border is not filtered (Section 5.1). Iterations are Jacobi.
//
// Each point is carried as its input position v0 plus a displacement d (both FP32, never
// summed into one float): v_j - v = (v0_j - v0) + (d_j - d), and the update only changes d.
// FP32 coordinates of 100 m carry ~4e-6 m of rounding, which the 1/|v_j - v| weights amplify
// near depth discontinuities; the displacement, millimetres to metres, rounds 1e3-1e5 times
// finer.
//
// One CTA owns a kLapTileH x kLapTileW tile of output points. It stages the tile plus a halo
// of (fused iterations x radius) points in shared memory -- v0 as three planes and d as a
// ping-pong pair of three planes -- and runs all fused iterations there (the valid region
// shrinks by the radius each iteration); each thread updates two vertically adjacent points,
// whose windows share most of their loads. An invalid point is staged as the finite
// sentinel kInvalidCoord: its difference to any real point is ~1e30, the squared distance
// overflows to +inf and rsqrt(+inf) = 0, so it carries no weight and no NaN enters a sum.
// HBM sees one read of the points (plus the previous displacement in later launches) and one
// write of the displacement per point per launch, however many iterations are fused.
#include <math.h>

#include "pl3d_internal.cuh"

namespace pl3d {
namespace {

struct LapAcc {
    float x, y, z, dx, dy, dz;   // centre: v0 and displacement
    float sx, sy, sz, ws;        // weighted sums
};

__device__ __forceinline__ void lap_begin(LapAcc& A, const float* V0, const float* D, int plane, int idx) {
    A.x = V0[idx];
    A.y = V0[plane + idx];
    A.z = V0[2 * plane + idx];
    A.dx = D[idx];
    A.dy = D[plane + idx];
    A.dz = D[2 * plane + idx];
    A.sx = A.sy = A.sz = A.ws = 0.f;
}

// Hardware reciprocal square root (PTX rsqrt.approx.ftz.f32, within 2 ulp): rsqrt(+inf) = 0.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One neighbour (Eq. 2): w = 1 / |v_j - v|; a neighbour at distance 0 is skipped.
__device__ __forceinline__ void lap_add(LapAcc& A, float xj, float yj, float zj, float dxj, float dyj, float dzj) {
    const float ex = (xj - A.x) + (dxj - A.dx);
    const float ey = (yj - A.y) + (dyj - A.dy);
    const float ez = (zj - A.z) + (dzj - A.dz);
    const float d2 = ex * ex + ey * ey + ez * ez;
    const float w = d2 > 0.f ? rsqrt_approx(d2) : 0.f;
    A.sx = fmaf(w, ex, A.sx);
    A.sy = fmaf(w, ey, A.sy);
    A.sz = fmaf(w, ez, A.sz);
    A.ws += w;
}

template <int R>
__global__ void __launch_bounds__(kLapThreads) lap_smooth_kernel(LapArgs a) {
    extern __shared__ float smem[];
    constexpr int TH = kLapTileH, TW = kLapTileW;
    const int halo = a.iters * R;
    const int RH = TH + 2 * halo;
    const int RW = TW + 2 * halo;
    const int plane = (RH + 1) * RW;           // one spare row: a strip's second point never reads past it
    float* V0 = smem;                          // [3][plane], read-only after staging
    float* cur = smem + 3 * plane;             // [3][plane] displacement
    float* nxt = smem + 6 * plane;             // [3][plane] displacement
    const int u0 = blockIdx.y * TH - halo;
    const int v0c = blockIdx.x * TW - halo;
    const int H = a.H, W = a.W;

    for (int i = threadIdx.x; i < RH * RW; i += blockDim.x) {
        const int r = i / RW, c = i - r * RW;
        const int gu = u0 + r, gv = v0c + c;
        float x = kInvalidCoord, y = kInvalidCoord, z = kInvalidCoord, dx = 0.f, dy = 0.f, dz = 0.f;
        if (gu >= 0 && gu < H && gv >= 0 && gv < W) {
            const size_t p = (size_t)gu * W + gv;
            const float px = __ldg(a.points + 3 * p), py = __ldg(a.points + 3 * p + 1),
                        pz = __ldg(a.points + 3 * p + 2);
            if (point_valid(px, py, pz)) {
                x = px;
                y = py;
                z = pz;
                if (a.in_dx) {
                    dx = __ldg(a.in_dx + p);
                    dy = __ldg(a.in_dy + p);
                    dz = __ldg(a.in_dz + p);
                }
            }
        }
        V0[i] = x;
        V0[plane + i] = y;
        V0[2 * plane + i] = z;
        cur[i] = dx;
        cur[plane + i] = dy;
        cur[2 * plane + i] = dz;
    }
    __syncthreads();

    for (int t = 1; t <= a.iters; ++t) {
        const int lo = t * R;
        const int ch = RH - 2 * lo, cw = RW - 2 * lo;
        const int strips = (ch + 1) >> 1;
        for (int i = threadIdx.x; i < strips * cw; i += blockDim.x) {
            const int sr = i / cw;
            const int r = lo + 2 * sr, c = lo + (i - sr * cw);
            const bool two = r + 1 < RH - lo;
            const int idxA = r * RW + c, idxB = idxA + RW;
            const int gu = u0 + r, gv = v0c + c;
            const bool colpin = gv < R || gv >= W - R;
            // Both points are always computed (a missing second point reads the spare row and
            // is not stored), so the unrolled window below has no data-dependent branch.
            LapAcc A, B;
            lap_begin(A, V0, cur, plane, idxA);
            lap_begin(B, V0, cur, plane, idxB);
#pragma unroll
            for (int dr = -R; dr <= R + 1; ++dr) {
#pragma unroll
                for (int dc = -R; dc <= R; ++dc) {
                    const bool forA = dr <= R && !(dr == 0 && dc == 0);
                    const bool forB = dr >= 1 - R && !(dr == 1 && dc == 0);
                    const int j = idxA + dr * RW + dc;
                    const float xj = V0[j], yj = V0[plane + j], zj = V0[2 * plane + j];
                    const float dxj = cur[j], dyj = cur[plane + j], dzj = cur[2 * plane + j];
                    if (forA) lap_add(A, xj, yj, zj, dxj, dyj, dzj);
                    if (forB) lap_add(B, xj, yj, zj, dxj, dyj, dzj);
                }
            }
            // Eq. 1 on the displacement; pinned border ring, invalid points and points without
            // a usable neighbour keep their displacement.
            const bool keepA = colpin || gu < R || gu >= H - R || A.x == kInvalidCoord || !(A.ws > 0.f);
            const float sA = keepA ? 0.f : __fdividef(a.lambda, A.ws);
            nxt[idxA] = fmaf(sA, A.sx, A.dx);
            nxt[plane + idxA] = fmaf(sA, A.sy, A.dy);
            nxt[2 * plane + idxA] = fmaf(sA, A.sz, A.dz);
            if (two) {
                const bool keepB = colpin || gu + 1 < R || gu + 1 >= H - R || B.x == kInvalidCoord || !(B.ws > 0.f);
                const float sB = keepB ? 0.f : __fdividef(a.lambda, B.ws);
                nxt[idxB] = fmaf(sB, B.sx, B.dx);
                nxt[plane + idxB] = fmaf(sB, B.sy, B.dy);
                nxt[2 * plane + idxB] = fmaf(sB, B.sz, B.dz);
            }
        }
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }

    // Write the CTA's own tile.
    for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
        const int r = halo + i / TW, c = halo + i % TW;
        const int gu = u0 + r, gv = v0c + c;
        if (gu >= H || gv >= W) continue;
        const int idx = r * RW + c;
        const size_t p = (size_t)gu * W + gv;
        const float dx = cur[idx], dy = cur[plane + idx], dz = cur[2 * plane + idx];
        a.out_dx[p] = dx;
        a.out_dy[p] = dy;
        a.out_dz[p] = dz;
        if (a.out_aos) {
            const bool valid = V0[idx] != kInvalidCoord;
            a.out_aos[3 * p] = valid ? V0[idx] + dx : NAN;
            a.out_aos[3 * p + 1] = valid ? V0[plane + idx] + dy : NAN;
            a.out_aos[3 * p + 2] = valid ? V0[2 * plane + idx] + dz : NAN;
        }
    }
}

template <int R>
cudaError_t launch_r(const LapArgs& a, cudaStream_t s) {
    const size_t smem = laplacian_smem_bytes(R, a.iters);
    dim3 grid(div_up(a.W, kLapTileW), div_up(a.H, kLapTileH));
    lap_smooth_kernel<R><<<grid, kLapThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int R>
cudaError_t configure_r() {
    return cudaFuncSetAttribute(lap_smooth_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)laplacian_smem_bytes(R, kLapMaxHalo / R));
}

}  // namespace

cudaError_t laplacian_configure() {
    cudaError_t e = configure_r<1>();
    if (e == cudaSuccess) e = configure_r<2>();
    if (e == cudaSuccess) e = configure_r<3>();
    return e;
}

size_t laplacian_smem_bytes(int radius, int iters) {
    const size_t halo = (size_t)iters * radius;
    return 3u * 3u * (kLapTileH + 2 * halo + 1) * (kLapTileW + 2 * halo) * sizeof(float);
}

cudaError_t launch_laplacian(const LapArgs& a, int radius, cudaStream_t s) {
    switch (radius) {
        case 1: return launch_r<1>(a, s);
        case 2: return launch_r<2>(a, s);
        case 3: return launch_r<3>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pl3d

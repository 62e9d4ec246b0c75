// lap_smooth.cu -- Laplacian vertex smoothing on the implicit image grid (Eq. 1-2, Section 5.1).
//
// Update of a valid interior point v with the valid points v_j of its k x k window
// (itself and points at distance 0 excluded):
//     w_j = 1 / |v_j - v|                                 (Eq. 2)
//     v'  = v + lambda * sum_j w_j (v_j - v) / sum_j w_j  (Eq. 1, umbrella form)
// Invalid points stay NaN, points with no usable neighbour stay put, and the ring of width
// k/2 at the image border is not filtered (Section 5.1). Iterations are Jacobi.
//
// Each point is carried as its input position v0 plus a displacement d (both FP32, never
// summed into one float): v_j - v = (v0_j - v0) + (d_j - d), and the update only changes d.
// FP32 coordinates of 100 m carry ~4e-6 m of rounding, which the 1/|v_j - v| weights amplify
// near depth discontinuities; the displacement, millimetres to metres, rounds 1e3-1e5 times
// finer.
//
// One CTA owns a kLapTileH x kLapTileW tile of output points. It stages the tile plus a
// halo of (fused iterations x radius) points in shared memory -- v0 as three planes and d as
// a ping-pong pair of three planes -- runs all fused iterations there (the valid region
// shrinks by the radius each iteration) and writes only its own tile's displacements. HBM
// sees one read of the points (plus the previous displacement in later launches) and one
// write of the displacement per point per launch, however many iterations are fused.
#include <math.h>

#include "pl3d_internal.cuh"

namespace pl3d {
namespace {

template <int R>
__global__ void __launch_bounds__(kLapThreads) lap_smooth_kernel(LapArgs a) {
    extern __shared__ float smem[];
    const int halo = a.iters * R;
    const int RH = kLapTileH + 2 * halo;
    const int RW = kLapTileW + 2 * halo;
    const int plane = RH * RW;
    const float* V0 = smem;                    // [3][plane], read-only after staging
    float* cur = smem + 3 * plane;             // [3][plane] displacement
    float* nxt = smem + 6 * plane;             // [3][plane] displacement
    const int u0 = blockIdx.y * kLapTileH - halo;
    const int v0c = blockIdx.x * kLapTileW - halo;
    const int H = a.H, W = a.W;

    // Stage the tile and its halo; any point with a non-finite coordinate becomes NaN.
    {
        float* V = smem;
        for (int i = threadIdx.x; i < plane; i += blockDim.x) {
            const int r = i / RW, c = i - r * RW;
            const int gu = u0 + r, gv = v0c + c;
            float x = NAN, y = NAN, z = NAN, dx = 0.f, dy = 0.f, dz = 0.f;
            if (gu >= 0 && gu < H && gv >= 0 && gv < W) {
                const size_t p = (size_t)gu * W + gv;
                x = __ldg(a.points + 3 * p);
                y = __ldg(a.points + 3 * p + 1);
                z = __ldg(a.points + 3 * p + 2);
                if (!(isfinite(x) && isfinite(y) && isfinite(z))) x = y = z = NAN;
                if (a.in_dx) {
                    dx = __ldg(a.in_dx + p);
                    dy = __ldg(a.in_dy + p);
                    dz = __ldg(a.in_dz + p);
                }
            }
            V[i] = x;
            V[plane + i] = y;
            V[2 * plane + i] = z;
            cur[i] = dx;
            cur[plane + i] = dy;
            cur[2 * plane + i] = dz;
        }
    }
    __syncthreads();

    for (int t = 1; t <= a.iters; ++t) {
        const int lo = t * R;
        const int ch = RH - 2 * lo, cw = RW - 2 * lo;
        for (int i = threadIdx.x; i < ch * cw; i += blockDim.x) {
            const int r = lo + i / cw, c = lo + i % cw;
            const int gu = u0 + r, gv = v0c + c;
            const int idx = r * RW + c;
            const float xi = V0[idx], yi = V0[plane + idx], zi = V0[2 * plane + idx];
            const float dxi = cur[idx], dyi = cur[plane + idx], dzi = cur[2 * plane + idx];
            const bool pinned = gu < R || gu >= H - R || gv < R || gv >= W - R;
            float ox = dxi, oy = dyi, oz = dzi;
            if (!pinned && xi == xi) {
                float sx = 0.f, sy = 0.f, sz = 0.f, ws = 0.f;
#pragma unroll
                for (int du = -R; du <= R; ++du) {
#pragma unroll
                    for (int dv = -R; dv <= R; ++dv) {
                        if (du == 0 && dv == 0) continue;
                        const int j = idx + du * RW + dv;
                        const float ex = (V0[j] - xi) + (cur[j] - dxi);
                        const float ey = (V0[plane + j] - yi) + (cur[plane + j] - dyi);
                        const float ez = (V0[2 * plane + j] - zi) + (cur[2 * plane + j] - dzi);
                        const float d2 = ex * ex + ey * ey + ez * ez;
                        const bool ok = d2 > 0.f;          // false for NaN neighbours and d = 0
                        const float w = ok ? rsqrtf(d2) : 0.f;
                        sx += ok ? w * ex : 0.f;
                        sy += ok ? w * ey : 0.f;
                        sz += ok ? w * ez : 0.f;
                        ws += w;
                    }
                }
                if (ws > 0.f) {
                    const float s = a.lambda / ws;
                    ox = dxi + s * sx;
                    oy = dyi + s * sy;
                    oz = dzi + s * sz;
                }
            }
            nxt[idx] = ox;
            nxt[plane + idx] = oy;
            nxt[2 * plane + idx] = oz;
        }
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }

    // Write the CTA's own tile.
    for (int i = threadIdx.x; i < kLapTileH * kLapTileW; i += blockDim.x) {
        const int r = halo + i / kLapTileW, c = halo + i % kLapTileW;
        const int gu = u0 + r, gv = v0c + c;
        if (gu >= H || gv >= W) continue;
        const int idx = r * RW + c;
        const size_t p = (size_t)gu * W + gv;
        const float dx = cur[idx], dy = cur[plane + idx], dz = cur[2 * plane + idx];
        a.out_dx[p] = dx;
        a.out_dy[p] = dy;
        a.out_dz[p] = dz;
        if (a.out_aos) {
            a.out_aos[3 * p] = V0[idx] + dx;
            a.out_aos[3 * p + 1] = V0[plane + idx] + dy;
            a.out_aos[3 * p + 2] = V0[2 * plane + idx] + dz;
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
    return 3u * 3u * (kLapTileH + 2 * halo) * (kLapTileW + 2 * halo) * sizeof(float);
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

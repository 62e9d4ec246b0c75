// lap_smooth.cu -- Laplacian vertex smoothing on the implicit image grid (Eq. 1-2, Section 5.1).
//
// Update of a valid interior point v with the valid points v_j of its k x k window
// (itself and points at distance 0 excluded):
//     w_j = 1 / |v_j - v|                                 (Eq. 2)
//     v'  = v + lambda * sum_j w_j (v_j - v) / sum_j w_j  (Eq. 1, umbrella form)
// Invalid points stay NaN, points with no usable neighbour stay put, and the ring of width
// k/2 at the image border is not filtered (Section 5.1). Iterations are Jacobi.
//
// One CTA owns a kLapTileH x kLapTileW tile of output points. It stages the tile plus a
// halo of (fused iterations x radius) points in shared memory as three planes (x, y, z),
// runs all fused iterations there with a ping-pong pair of buffers (the valid region
// shrinks by the radius each iteration) and writes only its own tile. HBM sees one read
// and one write per point per launch however many iterations are fused.
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
    float* cur = smem;
    float* nxt = smem + 3 * plane;
    const int u0 = blockIdx.y * kLapTileH - halo;
    const int v0 = blockIdx.x * kLapTileW - halo;
    const int H = a.H, W = a.W;

    // Stage the tile and its halo; any point with a non-finite coordinate becomes NaN.
    for (int i = threadIdx.x; i < plane; i += blockDim.x) {
        const int r = i / RW, c = i - r * RW;
        const int gu = u0 + r, gv = v0 + c;
        float x = NAN, y = NAN, z = NAN;
        if (gu >= 0 && gu < H && gv >= 0 && gv < W) {
            const size_t p = (size_t)gu * W + gv;
            if (a.in_aos) {
                x = __ldg(a.in_aos + 3 * p);
                y = __ldg(a.in_aos + 3 * p + 1);
                z = __ldg(a.in_aos + 3 * p + 2);
            } else {
                x = __ldg(a.in_x + p);
                y = __ldg(a.in_y + p);
                z = __ldg(a.in_z + p);
            }
            if (!(isfinite(x) && isfinite(y) && isfinite(z))) x = y = z = NAN;
        }
        cur[i] = x;
        cur[plane + i] = y;
        cur[2 * plane + i] = z;
    }
    __syncthreads();

    for (int t = 1; t <= a.iters; ++t) {
        const int lo = t * R;
        const int ch = RH - 2 * lo, cw = RW - 2 * lo;
        for (int i = threadIdx.x; i < ch * cw; i += blockDim.x) {
            const int r = lo + i / cw, c = lo + i % cw;
            const int gu = u0 + r, gv = v0 + c;
            const int idx = r * RW + c;
            const float xi = cur[idx], yi = cur[plane + idx], zi = cur[2 * plane + idx];
            const bool pinned = gu < R || gu >= H - R || gv < R || gv >= W - R;
            float ox = xi, oy = yi, oz = zi;
            if (!pinned && xi == xi) {
                float sx = 0.f, sy = 0.f, sz = 0.f, ws = 0.f;
#pragma unroll
                for (int du = -R; du <= R; ++du) {
#pragma unroll
                    for (int dv = -R; dv <= R; ++dv) {
                        if (du == 0 && dv == 0) continue;
                        const int j = idx + du * RW + dv;
                        const float dx = cur[j] - xi;
                        const float dy = cur[plane + j] - yi;
                        const float dz = cur[2 * plane + j] - zi;
                        const float d2 = dx * dx + dy * dy + dz * dz;
                        const bool ok = d2 > 0.f;          // false for NaN neighbours and d = 0
                        const float w = ok ? rsqrtf(d2) : 0.f;
                        sx += ok ? w * dx : 0.f;
                        sy += ok ? w * dy : 0.f;
                        sz += ok ? w * dz : 0.f;
                        ws += w;
                    }
                }
                if (ws > 0.f) {
                    const float s = a.lambda / ws;
                    ox = xi + s * sx;
                    oy = yi + s * sy;
                    oz = zi + s * sz;
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
        const int gu = u0 + r, gv = v0 + c;
        if (gu >= H || gv >= W) continue;
        const int idx = r * RW + c;
        const size_t p = (size_t)gu * W + gv;
        const float x = cur[idx], y = cur[plane + idx], z = cur[2 * plane + idx];
        a.out_x[p] = x;
        a.out_y[p] = y;
        a.out_z[p] = z;
        if (a.out_aos) {
            a.out_aos[3 * p] = x;
            a.out_aos[3 * p + 1] = y;
            a.out_aos[3 * p + 2] = z;
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
    return 2u * 3u * (kLapTileH + 2 * halo) * (kLapTileW + 2 * halo) * sizeof(float);
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

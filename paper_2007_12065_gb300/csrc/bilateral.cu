// bilateral.cu -- triangle centroids and normals over T_FC (Section 5.2), bilateral normal
// filtering (Eq. 3-6), the triangle mask (Algorithm 1 + the edge predicate of Algorithm 4)
// and group assignment (Algorithm 4), fused in one kernel.
//
// Triangles of quad (u, v): first = {p3, p2, p1}, second = {p1, p4, p3} with p1 = (u, v),
// p2 = (u, v+1), p3 = (u+1, v+1), p4 = (u+1, v) (Algorithm 1); normal = (b - a) x (c - a)
// normalised, centroid = (a + b + c) / 3.
//
// Bilateral iteration (Jacobi), for a triangle i with a normal:
//     n_i' = normalize( sum_j W_c(|c_i - c_j|) W_s(|n_i - n_j|) n_j )      (Eq. 3; K cancels)
//     W_c = exp(-|c_i - c_j|^2 / (2 sigma_c^2)),  W_s = exp(-|n_i - n_j|^2 / (2 sigma_s^2))
// over both triangles of every quad in the k x k quad block centred on i's quad, i itself
// included, triangles outside the image or without a normal skipped. Both exponentials are
// folded into one exp2 with the scales precomputed on the host.
//
// Smoothed points arrive as input position v0 plus displacement d (see df32.cuh); edges are
// formed as exact float pairs and the cross product with error-free products, so the normal
// of a sliver triangle is as accurate as the pair allows rather than as FP32 coordinates do.
//
// One CTA owns kBilTileH x kBilTileW quads. It stages the smoothed points of its tile plus a
// halo of (fused iterations x radius) quads, builds centroids and normals of every staged
// triangle in shared memory, runs the fused iterations there (the valid region shrinks by
// the radius each iteration), and finishes its own quads: mask, normal, group, and the
// initial union-find parent (GID when grouped, -1 otherwise). When the iterations do not fit
// one launch's halo, non-final launches hand their normals to the next through an AoS carry
// buffer and final launches re-stage them.
//
// A triangle without a normal is stored as n = 0, c = kAbsentCentroid: against any real
// triangle its weight is exp2(-inf) = 0, so it drops out of every sum without a branch.
#include <math.h>

#include "df32.cuh"
#include "pl3d_internal.cuh"

namespace pl3d {
namespace {

struct V3 {
    float x, y, z;
};

__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// A staged point: input position and displacement.
struct SP {
    float x, y, z, dx, dy, dz;
};

__device__ __forceinline__ SP load_sp(const float* P, int pplane, int i) {
    return {P[i], P[pplane + i], P[2 * pplane + i], P[3 * pplane + i], P[4 * pplane + i], P[5 * pplane + i]};
}

// Unnormalised normal (b - a) x (c - a), each component rounded once from exact float pairs.
__device__ __forceinline__ V3 exact_cross(const SP& a, const SP& b, const SP& c) {
    const F2 e1x = pair_diff(a.x, a.dx, b.x, b.dx), e1y = pair_diff(a.y, a.dy, b.y, b.dy),
             e1z = pair_diff(a.z, a.dz, b.z, b.dz);
    const F2 e2x = pair_diff(a.x, a.dx, c.x, c.dx), e2y = pair_diff(a.y, a.dy, c.y, c.dy),
             e2z = pair_diff(a.z, a.dz, c.z, c.dz);
    return {pair_sub_round(pair_mul(e1y, e2z), pair_mul(e1z, e2y)),
            pair_sub_round(pair_mul(e1z, e2x), pair_mul(e1x, e2z)),
            pair_sub_round(pair_mul(e1x, e2y), pair_mul(e1y, e2x))};
}

// Squared length of b - a from exact float pairs.
__device__ __forceinline__ float exact_len2(const SP& a, const SP& b) {
    return pair_sq_round(pair_diff(a.x, a.dx, b.x, b.dx)) + pair_sq_round(pair_diff(a.y, a.dy, b.y, b.dy)) +
           pair_sq_round(pair_diff(a.z, a.dz, b.z, b.dz));
}

__device__ __forceinline__ V3 centroid3(const SP& a, const SP& b, const SP& c) {
    const float k = 1.f / 3.f;
    return {((a.x + b.x + c.x) + (a.dx + b.dx + c.dx)) * k, ((a.y + b.y + c.y) + (a.dy + b.dy + c.dy)) * k,
            ((a.z + b.z + c.z) + (a.dz + b.dz + c.dz)) * k};
}

template <int R, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kBilThreads) bilateral_kernel(BilArgs a) {
    extern __shared__ float smem[];
    const int halo = a.iters * R;
    const int RQH = kBilTileH + 2 * halo;      // staged quads
    const int RQW = kBilTileW + 2 * halo;
    const int PW = RQW + 1;                    // staged points
    const int pplane = (RQH + 1) * PW;
    const int nq = RQH * RQW;
    const int nt = 2 * nq;                     // staged triangles, index 2 q + k
    float* P = smem;                           // [6][RQH+1][RQW+1]: v0 x, y, z, d x, y, z
    float* Cs = P + 6 * pplane;                // [3][nt]
    float* N0 = Cs + 3 * nt;                   // [3][nt]
    float* N1 = N0 + 3 * nt;                   // [3][nt]
    const int H = a.H, W = a.W, Hq = H - 1, Wq = W - 1;
    const int qu0 = blockIdx.y * kBilTileH - halo;
    const int qv0 = blockIdx.x * kBilTileW - halo;

    for (int i = threadIdx.x; i < pplane; i += blockDim.x) {
        const int r = i / PW, c = i - r * PW;
        const int gu = qu0 + r, gv = qv0 + c;
        float x = NAN, y = NAN, z = NAN, dx = 0.f, dy = 0.f, dz = 0.f;
        if (gu >= 0 && gu < H && gv >= 0 && gv < W) {
            const size_t p = (size_t)gu * W + gv;
            x = __ldg(a.points + 3 * p);
            y = __ldg(a.points + 3 * p + 1);
            z = __ldg(a.points + 3 * p + 2);
            if (!(isfinite(x) && isfinite(y) && isfinite(z))) x = y = z = NAN;
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

    // Centroids and normals of every staged triangle.
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const int qr = q / RQW, qc = q - qr * RQW;
        const int gu = qu0 + qr, gv = qv0 + qc;
        const bool exists = gu >= 0 && gu < Hq && gv >= 0 && gv < Wq;
        const int i1 = qr * PW + qc, i2 = i1 + 1, i3 = i1 + PW + 1, i4 = i1 + PW;
        const SP p1 = load_sp(P, pplane, i1), p2 = load_sp(P, pplane, i2);
        const SP p3 = load_sp(P, pplane, i3), p4 = load_sp(P, pplane, i4);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const SP& va = k == 0 ? p3 : p1;
            const SP& vb = k == 0 ? p2 : p4;
            const SP& vc = k == 0 ? p1 : p3;
            V3 n = {0.f, 0.f, 0.f};
            V3 c = {kAbsentCentroid, kAbsentCentroid, kAbsentCentroid};
            bool has_normal = false;
            if (exists && va.x == va.x && vb.x == vb.x && vc.x == vc.x) {
                if (FIRST) {
                    const V3 cr = exact_cross(va, vb, vc);
                    const float len2 = dot(cr, cr);
                    if (len2 > kDegenerateLen2) {
                        const float inv = rsqrtf(len2);
                        n = {cr.x * inv, cr.y * inv, cr.z * inv};
                        has_normal = true;
                    }
                } else {
                    const size_t gid = 2 * ((size_t)gu * Wq + gv) + k;
                    const float nx = __ldg(a.carry_in + 3 * gid);
                    if (nx == nx) {
                        n = {nx, __ldg(a.carry_in + 3 * gid + 1), __ldg(a.carry_in + 3 * gid + 2)};
                        has_normal = true;
                    }
                }
                if (has_normal) c = centroid3(va, vb, vc);
            }
            const int t = 2 * q + k;
            Cs[t] = c.x;
            Cs[nt + t] = c.y;
            Cs[2 * nt + t] = c.z;
            N0[t] = n.x;
            N0[nt + t] = n.y;
            N0[2 * nt + t] = n.z;
        }
    }
    __syncthreads();

    // Fused bilateral iterations; one thread filters both triangles of a quad, which share
    // the same window.
    float* cur = N0;
    float* nxt = N1;
    const float na = a.neg_a, ns = a.neg_s;
    for (int it = 1; it <= a.iters; ++it) {
        const int lo = it * R;
        const int ch = RQH - 2 * lo, cw = RQW - 2 * lo;
        for (int i = threadIdx.x; i < ch * cw; i += blockDim.x) {
            const int qr = lo + i / cw, qc = lo + i % cw;
            const int q = qr * RQW + qc;
            const int t0 = 2 * q, t1 = t0 + 1;
            const V3 n0 = {cur[t0], cur[nt + t0], cur[2 * nt + t0]};
            const V3 n1 = {cur[t1], cur[nt + t1], cur[2 * nt + t1]};
            const V3 c0 = {Cs[t0], Cs[nt + t0], Cs[2 * nt + t0]};
            const V3 c1 = {Cs[t1], Cs[nt + t1], Cs[2 * nt + t1]};
            V3 s0 = {0.f, 0.f, 0.f}, s1 = {0.f, 0.f, 0.f};
#pragma unroll
            for (int du = -R; du <= R; ++du) {
#pragma unroll
                for (int dv = -R; dv <= R; ++dv) {
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const int j = 2 * (q + du * RQW + dv) + kk;
                        const V3 nj = {cur[j], cur[nt + j], cur[2 * nt + j]};
                        const V3 cj = {Cs[j], Cs[nt + j], Cs[2 * nt + j]};
                        const V3 dc0 = sub(c0, cj), dn0 = sub(n0, nj);
                        const V3 dc1 = sub(c1, cj), dn1 = sub(n1, nj);
                        const float w0 = exp2f(na * dot(dc0, dc0) + ns * dot(dn0, dn0));
                        const float w1 = exp2f(na * dot(dc1, dc1) + ns * dot(dn1, dn1));
                        s0.x += w0 * nj.x;
                        s0.y += w0 * nj.y;
                        s0.z += w0 * nj.z;
                        s1.x += w1 * nj.x;
                        s1.y += w1 * nj.y;
                        s1.z += w1 * nj.z;
                    }
                }
            }
            const bool h0 = n0.x != 0.f || n0.y != 0.f || n0.z != 0.f;
            const bool h1 = n1.x != 0.f || n1.y != 0.f || n1.z != 0.f;
            const float l0 = dot(s0, s0), l1 = dot(s1, s1);
            V3 o0 = n0, o1 = n1;
            if (h0 && l0 > 0.f) {
                const float inv = rsqrtf(l0);
                o0 = {s0.x * inv, s0.y * inv, s0.z * inv};
            }
            if (h1 && l1 > 0.f) {
                const float inv = rsqrtf(l1);
                o1 = {s1.x * inv, s1.y * inv, s1.z * inv};
            }
            nxt[t0] = o0.x;
            nxt[nt + t0] = o0.y;
            nxt[2 * nt + t0] = o0.z;
            nxt[t1] = o1.x;
            nxt[nt + t1] = o1.y;
            nxt[2 * nt + t1] = o1.z;
        }
        __syncthreads();
        float* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }

    // Own quads: hand the normals on, or finish them.
    for (int i = threadIdx.x; i < kBilTileH * kBilTileW; i += blockDim.x) {
        const int qr = halo + i / kBilTileW, qc = halo + i % kBilTileW;
        const int gu = qu0 + qr, gv = qv0 + qc;
        if (gu >= Hq || gv >= Wq) continue;
        const int q = qr * RQW + qc;
        const size_t gid0 = 2 * ((size_t)gu * Wq + gv);
        if (!LAST) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int t = 2 * q + k;
                const V3 n = {cur[t], cur[nt + t], cur[2 * nt + t]};
                const bool has = n.x != 0.f || n.y != 0.f || n.z != 0.f;
                float* o = a.carry_out + 3 * (gid0 + k);
                o[0] = has ? n.x : NAN;
                o[1] = has ? n.y : NAN;
                o[2] = has ? n.z : NAN;
            }
            continue;
        }
        const int i1 = qr * PW + qc, i2 = i1 + 1, i3 = i1 + PW + 1, i4 = i1 + PW;
        const SP p1 = load_sp(P, pplane, i1), p2 = load_sp(P, pplane, i2);
        const SP p3 = load_sp(P, pplane, i3), p4 = load_sp(P, pplane, i4);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const SP& va = k == 0 ? p3 : p1;
            const SP& vb = k == 0 ? p2 : p4;
            const SP& vc = k == 0 ? p1 : p3;
            const bool valid = va.x == va.x && vb.x == vb.x && vc.x == vc.x;   // Algorithm 1
            const float longest2 = fmaxf(exact_len2(va, vb), fmaxf(exact_len2(vb, vc), exact_len2(vc, va)));
            const bool kept = valid && longest2 <= a.max_edge2;                // Algorithm 4, l_max
            const int t = 2 * q + k;
            const V3 n = {cur[t], cur[nt + t], cur[2 * nt + t]};
            const bool has = n.x != 0.f || n.y != 0.f || n.z != 0.f;
            int g = PL3D_NO_GROUP;
            if (kept && has) {                                                  // Algorithm 4, ang_min
                float best = -1.0f;
                for (int j = 0; j < a.nd.K; ++j) {
                    const float s = n.x * a.nd.v[3 * j] + n.y * a.nd.v[3 * j + 1] + n.z * a.nd.v[3 * j + 2];
                    if (s > best) {
                        best = s;
                        g = j;
                    }
                }
                if (best < a.min_dot) g = PL3D_NO_GROUP;
            }
            const size_t gid = gid0 + k;
            a.out_mask[gid] = kept ? 1 : 0;
            float* o = a.out_normals + 3 * gid;
            o[0] = has ? n.x : NAN;
            o[1] = has ? n.y : NAN;
            o[2] = has ? n.z : NAN;
            a.out_groups[gid] = (uint8_t)g;
            a.out_labels[gid] = g != PL3D_NO_GROUP ? (int32_t)gid : -1;
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
    const size_t points = 6 * (rqh + 1) * (rqw + 1);
    const size_t tris = 2 * rqh * rqw;
    return (points + 3 * 3 * tris) * sizeof(float);
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

// label.cu -- planar segments: connected components of equal group over twin edges
// (Algorithm 5, with the twins of Algorithm 2).
//
// Two triangles are joined when they share an edge, both have the same group g != 255 and,
// if max_offset > 0, |n^d_g . (c_i - c_j)| <= max_offset. In T_FC the twins of the first
// triangle of quad (u, v) are the second triangles of quads (u, v), (u, v+1) and (u-1, v);
// every edge is therefore visited once, from the first triangle that owns it.
//
// Components come from a lock-free union-find over the label array (the caller's output
// buffer, initialised by the bilateral kernel to GID for grouped triangles and -1
// otherwise). A root is only ever linked below a smaller root (compare-and-swap on the
// larger root), so every component ends with its smallest GID as root -- the label the
// result defines -- whatever order the unions run in. Finding a root halves the path as it
// walks (each visited node is pointed at its grandparent, an ancestor, so concurrent walks
// stay valid).
#include "pl3d_internal.cuh"

namespace pl3d {
namespace {

__device__ __forceinline__ int find_root_halving(int32_t* L, int x) {
    volatile int32_t* vl = L;
    while (true) {
        const int p = vl[x];
        if (p == x) return x;
        const int gp = vl[p];
        if (gp == p) return p;
        vl[x] = gp;
        x = gp;
    }
}

__device__ __forceinline__ void unite(int32_t* L, int a, int b) {
    while (true) {
        a = find_root_halving(L, a);
        b = find_root_halving(L, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(L + b, b, a);
        if (old == b) return;
        b = old;    // b stopped being a root meanwhile; continue from its new parent
    }
}

// Centroid of triangle k of quad (u, v) from the smoothed points v0 + d (offset test only).
__device__ __forceinline__ void centroid(const LabelArgs& a, int u, int v, int k, float c[3]) {
    const int W = a.W;
    const size_t p1 = (size_t)u * W + v, p2 = p1 + 1, p3 = p1 + W + 1, p4 = p1 + W;
    const size_t ia = k == 0 ? p3 : p1, ib = k == 0 ? p2 : p4, ic = k == 0 ? p1 : p3;
    const float* P = a.points;
    const float* D[3] = {a.dx, a.dy, a.dz};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        c[m] = ((P[3 * ia + m] + P[3 * ib + m] + P[3 * ic + m]) + (D[m][ia] + D[m][ib] + D[m][ic])) * (1.f / 3.f);
    }
}

__device__ __forceinline__ bool offset_ok(const LabelArgs& a, int g, const float ci[3], int uj, int vj, int kj) {
    float cj[3];
    centroid(a, uj, vj, kj, cj);
    const float* n = a.nd.v + 3 * g;
    const float off = n[0] * (ci[0] - cj[0]) + n[1] * (ci[1] - cj[1]) + n[2] * (ci[2] - cj[2]);
    return fabsf(off) <= a.max_offset;
}

__global__ void label_union_kernel(LabelArgs a) {
    const int Wq = a.W - 1, Hq = a.H - 1;
    const long long nq = (long long)Hq * Wq;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(2 * q);
        if (a.sizes) {
            a.sizes[i] = 0;
            a.sizes[i + 1] = 0;
        }
        const int g = a.groups[i];
        if (g == PL3D_NO_GROUP) continue;
        const int u = (int)(q / Wq), v = (int)(q % Wq);
        const bool offs = a.max_offset > 0.f;
        float ci[3];
        if (offs) centroid(a, u, v, 0, ci);
        // diagonal twin: second triangle of the same quad
        if (a.groups[i + 1] == g && (!offs || offset_ok(a, g, ci, u, v, 1))) unite(a.labels, i, i + 1);
        // right twin: second triangle of quad (u, v+1)
        if (v + 1 < Wq) {
            const int j = i + 3;
            if (a.groups[j] == g && (!offs || offset_ok(a, g, ci, u, v + 1, 1))) unite(a.labels, i, j);
        }
        // top twin: second triangle of quad (u-1, v)
        if (u >= 1) {
            const int j = i - 2 * Wq + 1;
            if (a.groups[j] == g && (!offs || offset_ok(a, g, ci, u - 1, v, 1))) unite(a.labels, i, j);
        }
    }
}

// Every grouped triangle takes its root. Walks only read: the single write per entry comes
// from its own thread, and a walk that reads an entry already rewritten reads its root.
__global__ void label_flatten_kernel(LabelArgs a) {
    const long long n = 2LL * (a.H - 1) * (a.W - 1);
    volatile int32_t* L = a.labels;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int x = L[i];
        if (x < 0) continue;
        while (true) {
            const int p = L[x];
            if (p == x) break;
            x = p;
        }
        L[i] = x;
        if (a.sizes) atomicAdd(a.sizes + x, 1);
    }
}

// Algorithm 5 keeps a segment only when it has more than tri_min triangles.
__global__ void label_filter_kernel(LabelArgs a) {
    const long long n = 2LL * (a.H - 1) * (a.W - 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int l = a.labels[i];
        if (l >= 0 && a.sizes[l] <= a.min_triangles) a.labels[i] = -1;
    }
}

constexpr int kThreads = 256;

int grid_for(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (int)b;
}

}  // namespace

cudaError_t launch_label_union(const LabelArgs& a, cudaStream_t s) {
    label_union_kernel<<<grid_for((long long)(a.H - 1) * (a.W - 1)), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_label_flatten(const LabelArgs& a, cudaStream_t s) {
    label_flatten_kernel<<<grid_for(2LL * (a.H - 1) * (a.W - 1)), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_label_filter(const LabelArgs& a, cudaStream_t s) {
    label_filter_kernel<<<grid_for(2LL * (a.H - 1) * (a.W - 1)), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pl3d

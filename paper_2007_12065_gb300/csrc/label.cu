// label.cu -- planar segments across tile borders: connected components of equal group over
// twin edges (Algorithm 5, with the twins of Algorithm 2).
//
// Two triangles are joined when they share an edge, both have the same group g != 255 and,
// if max_offset > 0, |n^d_g . (c_i - c_j)| <= max_offset. In T_FC the twins of the first
// triangle of quad (u, v) are the second triangles of quads (u, v), (u, v+1) and (u-1, v);
// every edge is visited once, from the first triangle that owns it.
//
// The bilateral kernel has already joined every edge inside its tile and left each grouped
// triangle pointing at the GID of its tile-local root (the smallest GID of its tile-local
// component). What remains is:
//   label_merge_kernel    the edges that cross a tile border: the top edge of a tile's first
//                         quad row and the right edge of its last quad column. Union-find
//                         with min-index roots (uf.cuh), so labels are component minima
//                         whatever the order.
//   label_flatten_kernel  every grouped triangle takes its root; with tri_min > 0 it also
//                         counts segment sizes, one atomic per run of equal roots in a warp.
//   label_filter_kernel   (tri_min > 0) drops segments with at most tri_min triangles.
#include "pl3d_internal.cuh"
#include "uf.cuh"

namespace pl3d {
namespace {

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

__device__ __forceinline__ bool offset_ok(const LabelArgs& a, int g, int u, int v, int uj, int vj) {
    if (!(a.max_offset > 0.f)) return true;
    float ci[3], cj[3];
    centroid(a, u, v, 0, ci);
    centroid(a, uj, vj, 1, cj);
    const float* n = a.nd.v + 3 * g;
    const float off = n[0] * (ci[0] - cj[0]) + n[1] * (ci[1] - cj[1]) + n[2] * (ci[2] - cj[2]);
    return fabsf(off) <= a.max_offset;
}

// Work items: (rows - 1) tile-row borders x Wq quads, then (cols - 1) tile-column borders x Hq.
__global__ void label_merge_kernel(LabelArgs a) {
    const int Wq = a.W - 1, Hq = a.H - 1;
    const int rb = div_up(Hq, a.tile_h) - 1;
    const int cb = div_up(Wq, a.tile_w) - 1;
    const long long n_row_items = (long long)rb * Wq;
    const long long n = n_row_items + (long long)cb * Hq;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < n; w += (long long)gridDim.x * blockDim.x) {
        int u, v, uj, vj;
        if (w < n_row_items) {           // top edge of the first quad row of a tile
            u = (int)(w / Wq + 1) * a.tile_h;
            v = (int)(w % Wq);
            uj = u - 1;
            vj = v;
        } else {                         // right edge of the last quad column of a tile
            const long long x = w - n_row_items;
            v = (int)(x / Hq + 1) * a.tile_w - 1;
            u = (int)(x % Hq);
            uj = u;
            vj = v + 1;
        }
        const int i = 2 * (u * Wq + v);
        const int j = 2 * (uj * Wq + vj) + 1;
        const int g = a.groups[i];
        if (g == PL3D_NO_GROUP || a.groups[j] != g) continue;
        if (!offset_ok(a, g, u, v, uj, vj)) continue;
        uf_unite(a.labels, i, j);
    }
}

// Every grouped triangle takes its root (walks only read: the single write per entry comes
// from its own thread, and a walk that meets an entry already rewritten reads its root).
__global__ void label_flatten_kernel(LabelArgs a) {
    const long long n = 2LL * (a.H - 1) * (a.W - 1);
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_iter = (n + stride - 1) / stride;
    const long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long it = 0; it < n_iter; ++it) {          // uniform trip count: whole warps stay together
        const long long i = base + it * stride;
        int root = -1;
        if (i < n && a.labels[i] >= 0) {
            root = uf_root(a.labels, (int)i);
            a.labels[i] = root;
        }
        if (a.sizes) {
            const unsigned peers = __match_any_sync(0xffffffffu, root);
            const int leader = __ffs(peers) - 1;
            if (root >= 0 && (int)(threadIdx.x & 31) == leader) atomicAdd(a.sizes + root, __popc(peers));
        }
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

cudaError_t launch_label_merge(const LabelArgs& a, cudaStream_t s) {
    const int Wq = a.W - 1, Hq = a.H - 1;
    const long long n = (long long)(div_up(Hq, a.tile_h) - 1) * Wq + (long long)(div_up(Wq, a.tile_w) - 1) * Hq;
    label_merge_kernel<<<grid_for(n > 0 ? n : 1), kThreads, 0, s>>>(a);
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

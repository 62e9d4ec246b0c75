// pl3d_fastga.cu -- the Fast Gaussian Accumulator (Section 6) on the device: the histogram of
// triangle normals over the cells of a refined icosahedron, and peak detection on the host.
//
// Cells (Section 6.1.1). Level 0 is the icosahedron with the 12 vertices (-1, phi, 0),
// (1, phi, 0), (-1, -phi, 0), (1, -phi, 0), (0, -1, phi), (0, 1, phi), (0, -1, -phi),
// (0, 1, -phi), (phi, 0, -1), (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1) (unit length, this order)
// and the 20 faces formed by the triples of mutually adjacent vertices, in lexicographic order of
// the sorted triple, oriented counter-clockwise from outside. Level l + 1 splits face p = (a, b, c)
// into faces 4p .. 4p + 3 = (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca), the midpoints
// projected onto the sphere. A cell's surface normal is its flat face's unit normal.
//
// Search (Section 6.1.3, Algorithm 3). The paper narrows the search with a space-filling-curve
// id, an interpolated window and a binary search, then compares the cell found with its 12
// neighbours. Here the first stage is a descent of the refinement: the level-0 face with the
// closest normal, then at each level the child containing the normal -- the children of a face
// tile its spherical triangle exactly, and three inner edge planes tell them apart. The nearest surface normal is then taken over
// that cell and its 1-ring neighbours (cells sharing a vertex), as in Algorithm 3; the nearest
// cell always lies there (checked on dense random samples at levels 3 and 4).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "pl3d_ctx.cuh"

namespace pl3d {
namespace fastga {

constexpr int kMaxLevel = 5;
constexpr int kNbrs = 12;

// Host-built tables of one refinement level (device copies live in the context).
struct Tables {
    int level = -1;
    int cells = 0;
    float face0[60];                  // unit normals of the 20 faces of level 0
    std::vector<float> split_planes;  // per face of levels 0..level-1: its 3 inner edge planes (9 floats)
    std::vector<int> level_offset;    // first face of each level in split_planes
    std::vector<float> normals;       // [cells][3] surface normals of the last level
    std::vector<int32_t> nbrs;        // [cells][12] 1-ring neighbours, ascending, -1 padded
};

struct V3d {
    double x, y, z;
};

V3d sub(V3d a, V3d b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3d crs(V3d a, V3d b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V3d unit(V3d a) {
    const double l = sqrt(a.x * a.x + a.y * a.y + a.z * a.z);
    return {a.x / l, a.y / l, a.z / l};
}
double det3(V3d a, V3d b, V3d c) { return a.x * (b.y * c.z - b.z * c.y) - a.y * (b.x * c.z - b.z * c.x) + a.z * (b.x * c.y - b.y * c.x); }

Tables build(int level) {
    const double phi = (1.0 + sqrt(5.0)) / 2.0;
    const double raw[12][3] = {{-1, phi, 0}, {1, phi, 0}, {-1, -phi, 0}, {1, -phi, 0}, {0, -1, phi}, {0, 1, phi},
                               {0, -1, -phi}, {0, 1, -phi}, {phi, 0, -1}, {phi, 0, 1}, {-phi, 0, -1}, {-phi, 0, 1}};
    std::vector<V3d> V;
    for (auto& r : raw) V.push_back(unit({r[0], r[1], r[2]}));
    auto dist2 = [&](int i, int j) {
        const double dx = raw[i][0] - raw[j][0], dy = raw[i][1] - raw[j][1], dz = raw[i][2] - raw[j][2];
        return dx * dx + dy * dy + dz * dz;
    };
    std::vector<std::array<int, 3>> F;
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j)
            for (int k = j + 1; k < 12; ++k)
                if (fabs(dist2(i, j) - 4) < 1e-9 && fabs(dist2(j, k) - 4) < 1e-9 && fabs(dist2(i, k) - 4) < 1e-9) {
                    const V3d a = {raw[i][0], raw[i][1], raw[i][2]}, b = {raw[j][0], raw[j][1], raw[j][2]},
                              c = {raw[k][0], raw[k][1], raw[k][2]};
                    if (det3(a, b, c) > 0) F.push_back({i, j, k});
                    else F.push_back({i, k, j});
                }
    Tables t;
    t.level = level;
    for (int i = 0; i < 20; ++i) {
        const V3d n = unit(crs(sub(V[F[i][1]], V[F[i][0]]), sub(V[F[i][2]], V[F[i][0]])));
        t.face0[3 * i] = (float)n.x;
        t.face0[3 * i + 1] = (float)n.y;
        t.face0[3 * i + 2] = (float)n.z;
    }
    for (int l = 0; l < level; ++l) {
        t.level_offset.push_back((int)(t.split_planes.size() / 9));
        std::map<std::pair<int, int>, int> mid;
        auto midpoint = [&](int a, int b) {
            const std::pair<int, int> key(std::min(a, b), std::max(a, b));
            auto it = mid.find(key);
            if (it != mid.end()) return it->second;
            const V3d p = unit({V[a].x + V[b].x, V[a].y + V[b].y, V[a].z + V[b].z});
            V.push_back(p);
            mid[key] = (int)V.size() - 1;
            return (int)V.size() - 1;
        };
        std::vector<std::array<int, 3>> nf;
        nf.reserve(F.size() * 4);
        for (const auto& f : F) {
            const int a = f[0], b = f[1], c = f[2];
            const int ab = midpoint(a, b), bc = midpoint(b, c), ca = midpoint(c, a);
            // the inner edges cutting off the corner children 0 (at a), 1 (at b), 2 (at c): a normal
            // of the face on the positive side of plane j lies in child j, on no positive side in
            // the middle child 3
            const V3d planes[3] = {unit(crs(V[ab], V[ca])), unit(crs(V[bc], V[ab])), unit(crs(V[ca], V[bc]))};
            for (const V3d& p : planes) {
                t.split_planes.push_back((float)p.x);
                t.split_planes.push_back((float)p.y);
                t.split_planes.push_back((float)p.z);
            }
            nf.push_back({a, ab, ca});
            nf.push_back({ab, b, bc});
            nf.push_back({ca, bc, c});
            nf.push_back({ab, bc, ca});
        }
        F.swap(nf);
    }
    t.cells = (int)F.size();
    for (const auto& f : F) {
        const V3d n = unit(crs(sub(V[f[1]], V[f[0]]), sub(V[f[2]], V[f[0]])));
        t.normals.push_back((float)n.x);
        t.normals.push_back((float)n.y);
        t.normals.push_back((float)n.z);
    }
    std::vector<std::vector<int>> inc(V.size());
    for (int i = 0; i < t.cells; ++i)
        for (int v : F[i]) inc[v].push_back(i);
    t.nbrs.assign((size_t)t.cells * kNbrs, -1);
    for (int i = 0; i < t.cells; ++i) {
        std::vector<int> nb;
        for (int v : F[i])
            for (int j : inc[v])
                if (j != i) nb.push_back(j);
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        for (size_t k = 0; k < nb.size() && k < (size_t)kNbrs; ++k) t.nbrs[(size_t)i * kNbrs + k] = nb[k];
    }
    return t;
}

const Tables& tables(int level) {
    static std::mutex mu;
    static Tables cache[kMaxLevel + 1];
    std::lock_guard<std::mutex> lock(mu);
    if (cache[level].level != level) cache[level] = build(level);
    return cache[level];
}

struct GaArgs {
    const float* normals;     // [n][3]
    const uint8_t* mask;      // [n] or nullptr
    long long n;
    int stride;
    int level;
    int cells;
    float face0[60];          // level-0 face normals (kernel parameter space: a broadcast read)
    const float* planes;      // split planes of the faces of levels 0..level-1
    const int* level_offset;  // [level]
    const float* cell_n;      // [cells][3]
    const int* nbrs;          // [cells][12]
    int* counts;              // [cells], zeroed before the launch
    int* out_cell;            // [n] or nullptr
};

__global__ void __launch_bounds__(kThreads) fastga_kernel(const __grid_constant__ GaArgs a) {
    extern __shared__ int hist[];   // [cells] private histogram of this CTA
    for (int i = threadIdx.x; i < a.cells; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    const long long n_samples = (a.n + a.stride - 1) / a.stride;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const long long n_iter = (n_samples + gstride - 1) / gstride;   // uniform: whole warps stay together
    for (long long it = 0; it < n_iter; ++it) {
        const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x + it * gstride;
        const bool in_range = s < n_samples;
        const long long i = in_range ? s * a.stride : 0;
        int cell = -1;
        float x = NAN, y = NAN, z = NAN;
        if (in_range) {
            x = __ldg(a.normals + 3 * i);
            y = __ldg(a.normals + 3 * i + 1);
            z = __ldg(a.normals + 3 * i + 2);
        }
        const bool use =
            in_range && (!a.mask || __ldg(a.mask + i) != 0) && isfinite(x) && isfinite(y) && isfinite(z);
        if (use) {
            // descent. Level 0: the face whose normal is closest (for the regular icosahedron each
            // face's spherical triangle is exactly the set of directions closest to its normal).
            int f = 0;
            float best = x * a.face0[0] + y * a.face0[1] + z * a.face0[2];
            for (int k = 1; k < 20; ++k) {
                const float v = x * a.face0[3 * k] + y * a.face0[3 * k + 1] + z * a.face0[3 * k + 2];
                if (v > best) {
                    best = v;
                    f = k;
                }
            }
            // every further level: the corner child on whose side of its inner edge the normal
            // lies, else the middle child (the four children tile the face exactly)
            for (int l = 0; l < a.level; ++l) {
                const float* p = a.planes + 9 * ((long long)__ldg(a.level_offset + l) + f);
                const float s0 = x * __ldg(p) + y * __ldg(p + 1) + z * __ldg(p + 2);
                const float s1 = x * __ldg(p + 3) + y * __ldg(p + 4) + z * __ldg(p + 5);
                const float s2 = x * __ldg(p + 6) + y * __ldg(p + 7) + z * __ldg(p + 8);
                int c = 3;
                float m = 0.f;
                if (s0 > m) m = s0, c = 0;
                if (s1 > m) m = s1, c = 1;
                if (s2 > m) m = s2, c = 2;
                f = 4 * f + c;
            }
            // Algorithm 3's local search: the closest surface normal among f and its neighbours
            cell = f;
            float bd = x * __ldg(a.cell_n + 3 * f) + y * __ldg(a.cell_n + 3 * f + 1) + z * __ldg(a.cell_n + 3 * f + 2);
            for (int k = 0; k < kNbrs; ++k) {
                const int j = __ldg(a.nbrs + kNbrs * f + k);
                if (j < 0) continue;
                const float d =
                    x * __ldg(a.cell_n + 3 * j) + y * __ldg(a.cell_n + 3 * j + 1) + z * __ldg(a.cell_n + 3 * j + 2);
                if (d > bd) {
                    bd = d;
                    cell = j;
                }
            }
        }
        // one shared-memory atomic per distinct cell in the warp: most normals of a scene fall in
        // the few cells of its dominant planes
        const unsigned peers = __match_any_sync(0xffffffffu, cell);
        if (cell >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(hist + cell, __popc(peers));
        if (a.out_cell && in_range) a.out_cell[i] = cell;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.cells; i += blockDim.x)
        if (hist[i]) atomicAdd(a.counts + i, hist[i]);
}

}  // namespace fastga
}  // namespace pl3d

using namespace pl3d;
using namespace pl3d::ctxutil;

extern "C" {

int pl3d_fastga_cells(int level, float* out_normals, int32_t* out_neighbors) {
    if (level < 0 || level > fastga::kMaxLevel) return PL3D_ERR_INVALID_ARG;
    const fastga::Tables& t = fastga::tables(level);
    if (out_normals) memcpy(out_normals, t.normals.data(), t.normals.size() * sizeof(float));
    if (out_neighbors) memcpy(out_neighbors, t.nbrs.data(), t.nbrs.size() * sizeof(int32_t));
    return t.cells;
}

int pl3d_fastga(pl3d_ctx* ctx, const float* normals, const uint8_t* mask, int64_t n, int level, int stride,
                int32_t* out_counts, int32_t* out_cells, void* stream) {
    if (!ctx || !normals || !out_counts || n < 0 || level < 0 || level > fastga::kMaxLevel || stride < 1)
        return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const fastga::Tables& t = fastga::tables(level);
    // device copies of the level's tables, kept by the context
    if (ctx->ga_level != level) {
        if (ctx->ga_tables && cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
        cudaFree(ctx->ga_tables);
        ctx->ga_tables = nullptr;
        ctx->ga_level = -1;
        const size_t b0 = t.split_planes.size() * 4, b1 = t.level_offset.size() * 4, b2 = t.normals.size() * 4,
                     b3 = t.nbrs.size() * 4;
        const size_t o1 = (b0 + 255) / 256 * 256, o2 = o1 + (b1 + 255) / 256 * 256, o3 = o2 + (b2 + 255) / 256 * 256;
        if (cudaMalloc((void**)&ctx->ga_tables, o3 + b3) != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_OUT_OF_MEMORY;
        }
        if (cudaMemcpy(ctx->ga_tables, t.split_planes.data(), b0, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->ga_tables + o1, t.level_offset.data(), b1, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->ga_tables + o2, t.normals.data(), b2, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->ga_tables + o3, t.nbrs.data(), b3, cudaMemcpyHostToDevice) != cudaSuccess)
            return PL3D_ERR_CUDA;
        ctx->ga_level = level;
        ctx->ga_off[0] = 0;
        ctx->ga_off[1] = o1;
        ctx->ga_off[2] = o2;
        ctx->ga_off[3] = o3;
    }
    if (cudaMemsetAsync(out_counts, 0, (size_t)t.cells * sizeof(int32_t), s) != cudaSuccess) return PL3D_ERR_CUDA;
    // triangles the stride skips are never visited: they read -1 (every byte 0xff)
    if (out_cells && stride > 1 && cudaMemsetAsync(out_cells, 0xff, (size_t)n * sizeof(int32_t), s) != cudaSuccess)
        return PL3D_ERR_CUDA;
    if (n == 0) return PL3D_OK;
    fastga::GaArgs a;
    a.normals = normals;
    a.mask = mask;
    a.n = n;
    a.stride = stride;
    a.level = level;
    a.cells = t.cells;
    memcpy(a.face0, t.face0, sizeof(a.face0));
    a.planes = reinterpret_cast<const float*>(ctx->ga_tables + ctx->ga_off[0]);
    a.level_offset = reinterpret_cast<const int*>(ctx->ga_tables + ctx->ga_off[1]);
    a.cell_n = reinterpret_cast<const float*>(ctx->ga_tables + ctx->ga_off[2]);
    a.nbrs = reinterpret_cast<const int*>(ctx->ga_tables + ctx->ga_off[3]);
    a.counts = out_counts;
    a.out_cell = out_cells;
    const size_t smem = (size_t)t.cells * sizeof(int);
    const void* fn = reinterpret_cast<const void*>(&fastga::fastga_kernel);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PL3D_ERR_CUDA;
    const long long samples = (n + stride - 1) / stride;
    const int grid = persistent_grid(fn, smem, dev, Tuning{0, 0, 0}, (samples + kThreads - 1) / kThreads);
    if (grid <= 0) return PL3D_ERR_CUDA;
    cudaEvent_t e0, e1;
    record_start(ctx, s, &e0, &e1);
    void* args[1] = {&a};
    if (cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, smem, s) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    record_stop(ctx, s, kSlotFastga, e0, e1);
    ctx->launches += 1;
    return PL3D_OK;
}

int pl3d_fastga_peaks(int level, const int32_t* counts, float v_min, float d_peak, int max_peaks, float* out_normals,
                      int64_t* out_weights) {
    if (level < 0 || level > fastga::kMaxLevel || !counts || max_peaks < 0 || (max_peaks > 0 && !out_normals) ||
        !isfinite(v_min) || !isfinite(d_peak))
        return PL3D_ERR_INVALID_ARG;
    const fastga::Tables& t = fastga::tables(level);
    // a peak: count above v_min, not below any 1-ring neighbour (a plateau keeps its lowest index)
    std::vector<int> pk;
    for (int i = 0; i < t.cells; ++i) {
        if (!((float)counts[i] > v_min)) continue;
        bool peak = true;
        for (int k = 0; k < fastga::kNbrs && peak; ++k) {
            const int j = t.nbrs[(size_t)i * fastga::kNbrs + k];
            if (j >= 0 && !(counts[i] > counts[j] || (counts[i] == counts[j] && i < j))) peak = false;
        }
        if (peak) pk.push_back(i);
    }
    // single-linkage clusters of peaks closer than d_peak; each the count-weighted mean normal
    const int m = (int)pk.size();
    std::vector<int> parent(m);
    for (int i = 0; i < m; ++i) parent[i] = i;
    auto find = [&](int x) {
        while (parent[x] != x) x = parent[x];
        return x;
    };
    auto nrm = [&](int c, int d) { return (double)t.normals[3 * (size_t)c + d]; };
    for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j) {
            const double dx = nrm(pk[i], 0) - nrm(pk[j], 0), dy = nrm(pk[i], 1) - nrm(pk[j], 1),
                         dz = nrm(pk[i], 2) - nrm(pk[j], 2);
            if (sqrt(dx * dx + dy * dy + dz * dz) < d_peak) {
                const int ri = find(i), rj = find(j);
                if (ri != rj) parent[std::max(ri, rj)] = std::min(ri, rj);
            }
        }
    struct Cluster {
        double x = 0, y = 0, z = 0;
        int64_t w = 0;
        int first = 1 << 30;
    };
    std::map<int, Cluster> cl;
    for (int i = 0; i < m; ++i) {
        Cluster& c = cl[find(i)];
        const double w = counts[pk[i]];
        c.x += w * nrm(pk[i], 0);
        c.y += w * nrm(pk[i], 1);
        c.z += w * nrm(pk[i], 2);
        c.w += counts[pk[i]];
        c.first = std::min(c.first, pk[i]);
    }
    std::vector<Cluster> out;
    for (auto& kv : cl) out.push_back(kv.second);
    std::sort(out.begin(), out.end(), [](const Cluster& a, const Cluster& b) {
        return a.w != b.w ? a.w > b.w : a.first < b.first;
    });
    const int k = std::min((int)out.size(), max_peaks);
    for (int i = 0; i < k; ++i) {
        const double l = sqrt(out[i].x * out[i].x + out[i].y * out[i].y + out[i].z * out[i].z);
        out_normals[3 * i] = (float)(out[i].x / l);
        out_normals[3 * i + 1] = (float)(out[i].y / l);
        out_normals[3 * i + 2] = (float)(out[i].z / l);
        if (out_weights) out_weights[i] = out[i].w;
    }
    return k;
}

}  // extern "C"

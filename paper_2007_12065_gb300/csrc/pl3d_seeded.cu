// pl3d_seeded.cu -- Algorithm 5's region growing with the seed-relative point-to-plane limit
// (PL3D_FLAG_SEED_PTP), split between the GPU and the host.
//
// Algorithm 5 grows segments from seeds taken in GID order; a triangle joins the segment when
// it is reachable through twin half-edges over triangles of the seed's group that are in no
// segment yet, and its centroid lies within ptp_max of the plane through the seed's centroid
// with the group's dominant normal. That is order dependent, but a component of the
// order-independent labeling (same-group triangles connected through twins, labelled by their
// smallest GID) whose triangles all lie within ptp_max of its smallest triangle's plane is
// exactly one segment of Algorithm 5: its smallest GID is the first seed to reach it, and the
// seed's slab holds all of it. So:
//   1. the frame kernel labels the components (no offset test, no tri_min);
//   2. check_kernel flags every component with a triangle outside its root's slab and writes
//      each grouped triangle's centroid;
//   3. the host regrows only the flagged components, seeds in GID order, applies tri_min to
//      every segment and uploads the labels.
#include <math.h>
#include <string.h>

#include <vector>

#include "pl3d_ctx.cuh"

namespace pl3d {
namespace seeded {

struct CheckArgs {
    const float* points;
    const float* disp;       // final displacement of the frame (smoothed point = point + disp)
    const uint8_t* groups;
    const int32_t* labels;
    int H, W;
    float ptp;
    uint8_t* flags;          // [2Q] per root: 1 = some triangle of its component leaves the slab
    float* centroids;        // [2Q][3]
    Dominant nd;
};

__device__ __forceinline__ void centroid(const CheckArgs& a, long long gid, float c[3]) {
    const int Wq = a.W - 1;
    const long long q = gid >> 1, u = q / Wq, v = q - u * Wq;
    const long long p1 = u * a.W + v, p2 = p1 + 1, p3 = p1 + a.W + 1, p4 = p1 + a.W;
    const long long i0 = 3 * ((gid & 1) == 0 ? p3 : p1), i1 = 3 * ((gid & 1) == 0 ? p2 : p4),
                    i2 = 3 * ((gid & 1) == 0 ? p1 : p3);
    const float k = 1.f / 3.f;
    for (int d = 0; d < 3; ++d)
        c[d] = ((__ldg(a.points + i0 + d) + __ldg(a.points + i1 + d) + __ldg(a.points + i2 + d)) +
                (__ldcg(a.disp + i0 + d) + __ldcg(a.disp + i1 + d) + __ldcg(a.disp + i2 + d))) *
               k;
}

__global__ void __launch_bounds__(kThreads) check_kernel(const __grid_constant__ CheckArgs a) {
    const long long n = 2LL * (a.H - 1) * (a.W - 1);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int l = __ldcg(a.labels + i);
        if (l < 0) continue;
        float c[3], r[3];
        centroid(a, i, c);
        a.centroids[3 * i] = c[0];
        a.centroids[3 * i + 1] = c[1];
        a.centroids[3 * i + 2] = c[2];
        centroid(a, l, r);
        const float* d = a.nd.v + 3 * __ldcg(a.groups + i);
        if (fabsf(d[0] * (c[0] - r[0]) + d[1] * (c[1] - r[1]) + d[2] * (c[2] - r[2])) > a.ptp) a.flags[l] = 1;
    }
}

// Twins of triangle t (Algorithm 2): first (k = 0) -> right, top, its second; second -> left,
// bottom, its first.
int twins(long long t, int Hq, int Wq, long long out[3]) {
    const long long q = t >> 1, u = q / Wq, v = q - u * Wq;
    int m = 0;
    if ((t & 1) == 0) {
        if (v + 1 < Wq) out[m++] = 2 * (q + 1) + 1;
        if (u > 0) out[m++] = 2 * (q - Wq) + 1;
        out[m++] = 2 * q + 1;
    } else {
        if (v > 0) out[m++] = 2 * (q - 1);
        if (u + 1 < Hq) out[m++] = 2 * (q + Wq);
        out[m++] = 2 * q;
    }
    return m;
}

}  // namespace seeded

int seeded_labels(const FrameScratch& sc, const float* disp, const float* points, int H, int W, const pl3d_params* p,
                  const float* nd_host, int K, const uint8_t* groups, int32_t* labels, cudaStream_t s) {
    const long long n = 2LL * (H - 1) * (W - 1);
    seeded::CheckArgs a;
    memset(&a, 0, sizeof(a));
    a.points = points;
    a.disp = disp;
    a.groups = groups;
    a.labels = labels;
    a.H = H;
    a.W = W;
    a.ptp = p->max_offset;
    a.flags = sc.seed_flags;
    a.centroids = sc.seed_centroids;
    std::vector<double> nd(3 * (size_t)K);
    a.nd.K = K;
    for (int j = 0; j < K; ++j) {
        const double x = nd_host[3 * j], y = nd_host[3 * j + 1], z = nd_host[3 * j + 2];
        const double len = sqrt(x * x + y * y + z * z);
        nd[3 * j] = x / len;
        nd[3 * j + 1] = y / len;
        nd[3 * j + 2] = z / len;
        for (int d = 0; d < 3; ++d) a.nd.v[3 * j + d] = (float)nd[3 * j + d];
    }
    if (cudaMemsetAsync(sc.seed_flags, 0, (size_t)n, s) != cudaSuccess) return PL3D_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PL3D_ERR_CUDA;
    const void* fn = reinterpret_cast<const void*>(&seeded::check_kernel);
    const int grid = persistent_grid(fn, 0, dev, Tuning{0, 0, 0}, (n + kThreads - 1) / kThreads);
    if (grid <= 0) return PL3D_ERR_CUDA;
    void* args[1] = {&a};
    if (cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, 0, s) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    std::vector<int32_t> lab(n);
    std::vector<uint8_t> flag(n);
    if (cudaMemcpyAsync(lab.data(), labels, n * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(flag.data(), sc.seed_flags, n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PL3D_ERR_CUDA;
    bool any = false;
    for (long long i = 0; i < n && !any; ++i) any = flag[i] != 0;
    if (any) {
        // regrow the flagged components: seeds in GID order, the seed-relative slab
        std::vector<uint8_t> g(n);
        std::vector<float> c(3 * (size_t)n);
        if (cudaMemcpyAsync(g.data(), groups, n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(c.data(), sc.seed_centroids, 12 * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return PL3D_ERR_CUDA;
        const int Hq = H - 1, Wq = W - 1;
        std::vector<int32_t> out(lab);
        std::vector<uint8_t> todo(n, 0);
        for (long long i = 0; i < n; ++i)
            if (lab[i] >= 0 && flag[lab[i]]) todo[i] = 1;
        std::vector<long long> queue;
        const double ptp = p->max_offset;
        for (long long seed = 0; seed < n; ++seed) {
            if (!todo[seed]) continue;
            const double* d = nd.data() + 3 * g[seed];
            const float* cs = c.data() + 3 * seed;
            queue.clear();
            queue.push_back(seed);
            todo[seed] = 0;
            out[seed] = (int32_t)seed;
            for (size_t head = 0; head < queue.size(); ++head) {
                long long nb[3];
                const int m = seeded::twins(queue[head], Hq, Wq, nb);
                for (int k = 0; k < m; ++k) {
                    const long long j = nb[k];
                    if (!todo[j] || g[j] != g[seed]) continue;
                    const float* cj = c.data() + 3 * j;
                    const double off = fabs(d[0] * ((double)cj[0] - cs[0]) + d[1] * ((double)cj[1] - cs[1]) +
                                            d[2] * ((double)cj[2] - cs[2]));
                    if (off > ptp) continue;
                    todo[j] = 0;
                    out[j] = (int32_t)seed;
                    queue.push_back(j);
                }
            }
        }
        lab.swap(out);
    }
    // Algorithm 5 keeps a segment only when it has more than tri_min triangles
    if (p->min_triangles > 0) {
        std::vector<int32_t> size(n, 0);
        for (long long i = 0; i < n; ++i)
            if (lab[i] >= 0) ++size[lab[i]];
        for (long long i = 0; i < n; ++i)
            if (lab[i] >= 0 && size[lab[i]] <= p->min_triangles) lab[i] = -1;
    }
    if (any || p->min_triangles > 0) {
        if (cudaMemcpyAsync(labels, lab.data(), n * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return PL3D_ERR_CUDA;
    }
    return PL3D_OK;
}

}  // namespace pl3d

// frame_host.cu -- host side of the frame kernel: pass planning, TMA tensor maps, occupancy and
// the cooperative launch (which guarantees that every CTA of the grid is resident, as the grid
// barrier requires).
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "pl3d_internal.cuh"

namespace pl3d {

const void* frame_kernel_rb1(int rl);
const void* frame_kernel_rb2(int rl);
const void* frame_kernel_rb3(int rl);
const void* batch_kernel_rb1(int rl);
const void* batch_kernel_rb2(int rl);
const void* batch_kernel_rb3(int rl);

namespace {

const void* kernel_for(int rl, int rb) {
    switch (rb) {
        case 1: return frame_kernel_rb1(rl);
        case 2: return frame_kernel_rb2(rl);
        case 3: return frame_kernel_rb3(rl);
        default: return nullptr;
    }
}

const void* batch_kernel_for(int rl, int rb) {
    switch (rb) {
        case 1: return batch_kernel_rb1(rl);
        case 2: return batch_kernel_rb2(rl);
        case 3: return batch_kernel_rb3(rl);
        default: return nullptr;
    }
}

int round4(int n) { return (n + 3) & ~3; }

// Laplacian box: the tile, its halo and 3 spare rows for the 4-point strips that run past it.
BoxGeom lap_box(int halo, int tile_h) { return {tile_h + 2 * halo + 3, round4(3 * (kTile + 2 * halo) + 3)}; }
// Bilateral box: th x kTile quads, their halo, and one more row and column of points.
BoxGeom bil_box(int halo, int th) { return {th + 2 * halo + 1, round4(3 * (kTile + 2 * halo + 1) + 3)}; }

size_t bil_smem(int halo, int th) {
    const BoxGeom b = bil_box(halo, th);
    const int rq = kTile + 2 * halo, rh = th + 2 * halo;
    const int quads = align_floats(6 * (rh * rq + rq));
    const int boxes = 2 * align_floats(b.rows * b.cols);
    return 128 + 4 * (size_t)(2 * quads + (quads > boxes ? quads : boxes)) + 4 * (size_t)kTile * kTile +
           4 * (size_t)kExactCap;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// Tensor map of an AoS [H][W][3] float array as H rows of 3W floats; box = b. Out-of-bounds
// elements read as NaN (nan_fill) or zero.
bool encode_aos(CUtensorMap* map, const float* base, int H, int W, BoxGeom b, bool nan_fill) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)3 * W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)12 * W};
    const cuuint32_t box[2] = {(cuuint32_t)b.cols, (cuuint32_t)b.rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              nan_fill ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

void bilateral_scales(float sigma_c, float sigma_s, int iters, float* c_scale, float* a_norm) {
    const double log2e = 1.4426950408889634;
    double cs = 1.0, an = 0.0;
    if (iters > 0) {
        cs = sqrt(log2e / (2.0 * (double)sigma_c * (double)sigma_c));
        an = log2e / ((double)sigma_s * (double)sigma_s);
    }
    // finite and representable: c' = c * cs must not overflow for coordinates up to ~1e18
    *c_scale = (float)fmin(fmax(cs, 1e-18), 1e18);
    *a_norm = (float)fmin(an, 1e30);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

// Resident CTAs per device for a kernel and shared-memory size (cached).
namespace {
struct OccKey {
    const void* fn;
    size_t smem;
    int dev;
};
std::mutex g_occ_mutex;
OccKey g_occ_keys[64];
int g_occ_vals[64];
int g_occ_n = 0;
}  // namespace

int resident_ctas(const void* fn, size_t smem, int dev, int threads) {
    std::lock_guard<std::mutex> lock(g_occ_mutex);
    for (int i = 0; i < g_occ_n; ++i)
        if (g_occ_keys[i].fn == fn && g_occ_keys[i].smem == smem && g_occ_keys[i].dev == dev) return g_occ_vals[i];
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int v = per_sm * sms;
    if (g_occ_n < 64) {
        g_occ_keys[g_occ_n] = {fn, smem, dev};
        g_occ_vals[g_occ_n] = v;
        ++g_occ_n;
    }
    return v;
}

const void* batch_kernel_for_radii(int rl, int rb) { return batch_kernel_for(rl, rb); }

// Iterations per pass: as many as the halo allows, or fewer on request, but never so few that
// the passes outnumber kMaxPasses (a tuning must not turn a valid frame into an error).
static int fused_iters(int iters, int max_fuse, int requested) {
    int fuse = max_fuse;
    if (requested > 0 && requested < fuse) fuse = requested;
    const int least = (iters + kMaxPasses - 1) / kMaxPasses;
    return fuse < least ? least : fuse;
}

int lap_box_floats(int halo, int tile_h) {
    const BoxGeom b = lap_box(halo, tile_h);
    return align_floats(b.rows * b.cols);
}

size_t lap_smem_for(int box_floats, int stages, int dbufs) {
    return 128 + 4 * (size_t)(stages + dbufs) * box_floats;
}

int lap_stages_for(int box_floats, int dbufs) {
    int ns = kLapMaxStages;
    while (ns > 1 && lap_smem_for(box_floats, ns, dbufs) > (size_t)kTwoCtaSmem) --ns;
    return ns;
}

// A single-iteration first pass reads no displacement: taller tiles, one displacement buffer.
static bool lap_thin(int iters, bool first) { return first && iters == 1; }

// Tile height of a Laplacian pass: the tuning's, else 64 for a single-iteration first pass and 32
// otherwise; a height whose box and displacement buffers would not fit two CTAs per SM even
// without staging ahead falls back to 32.
static int lap_tile_h(int iters, bool first, int halo, int requested) {
    const bool thin = lap_thin(iters, first);
    const int dbufs = thin ? 1 : 2;
    const int th = requested > 0 ? requested : (thin ? kLapThinTileH : kTile);
    return lap_smem_for(lap_box_floats(halo, th), 1, dbufs) <= (size_t)kTwoCtaSmem ? th : kTile;
}

static int bil_tile_h(const Tuning& t) { return t.bil_tile_h > 0 ? t.bil_tile_h : kTile; }

size_t border_counters(int H, int W, const Tuning& t) {
    if (H < 2 || W < 2) return 0;
    return 2 * (size_t)div_up(H - 1, bil_tile_h(t)) * (size_t)div_up(W - 1, kTile);
}

const float* final_disp(const FrameScratch& sc, const pl3d_params* p, const Tuning& t) {
    const int rl = p->lap_iters > 0 ? p->lap_kernel / 2 : 1;
    const int lf = fused_iters(p->lap_iters, kLapMaxHalo / rl, t.lap_fuse);
    const int passes = p->lap_iters <= lf ? 1 : (p->lap_iters + lf - 1) / lf;   // as frame_build plans them
    return sc.disp[(passes - 1) & 1];
}

size_t frame_smem_bytes(const pl3d_params* p, const Tuning& t) {
    const int rl = p->lap_iters > 0 ? p->lap_kernel / 2 : 1;
    const int rb = p->bil_iters > 0 ? p->bil_kernel / 2 : 1;
    const int lf = fused_iters(p->lap_iters, kLapMaxHalo / rl, t.lap_fuse);
    const int bf = fused_iters(p->bil_iters, kBilMaxHalo / rb, t.bil_fuse);
    // the first pass of each filter fuses the most iterations, so it has the largest halo
    const int li = p->lap_iters < lf ? p->lap_iters : lf;
    const int lh = li * rl;
    const bool thin = lap_thin(li, true);
    const int ld = thin ? 1 : 2;
    const int lb = lap_box_floats(lh, lap_tile_h(li, true, lh, t.lap_tile_h));
    const size_t l = lap_smem_for(lb, lap_stages_for(lb, ld), ld);   // an upper bound: several stages need TMA
    const size_t b = bil_smem((p->bil_iters < bf ? p->bil_iters : bf) * rb, bil_tile_h(t));
    return l > b ? l : b;
}

int bilateral_passes(const pl3d_params* p, const Tuning& t) {
    const int br = p->bil_iters > 0 ? p->bil_kernel / 2 : 1;
    const int fuse = fused_iters(p->bil_iters, kBilMaxHalo / br, t.bil_fuse);
    return p->bil_iters <= fuse ? 1 : (p->bil_iters + fuse - 1) / fuse;
}

cudaError_t frame_configure() {
    const int lb = lap_box_floats(kLapMaxHalo, kTile), lt = lap_box_floats(1 * 3, kLapThinTileH);
    const size_t lap_need = std::max(lap_smem_for(lb, lap_stages_for(lb, 2), 2), lap_smem_for(lt, lap_stages_for(lt, 1), 1));
    const size_t need = std::max({lap_need, (size_t)kTwoCtaSmem, bil_smem(kBilMaxHalo, kTile)});
    for (int rl = 1; rl <= 3; ++rl)
        for (int rb = 1; rb <= 3; ++rb)
            for (const void* fn : {kernel_for(rl, rb), batch_kernel_for(rl, rb)}) {
                cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
                // all of the unified L1 / shared storage as shared memory, so that two CTAs fit per SM
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             cudaSharedmemCarveoutMaxShared);
                if (e != cudaSuccess) return e;
            }
    // the single-iteration Laplacian keeps its rings in static shared memory: all of it as shared
    // memory, so that its CTAs fit as many per SM as their registers allow
    for (bool with_d : {false, true}) {
        cudaError_t e = cudaFuncSetAttribute(lap1_kernel_for(with_d), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)lap1_smem_bytes(with_d));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(lap1_kernel_for(with_d), cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int frame_build(FrameArgs& a, FramePlan& plan, const FrameScratch& sc, const float* points, int H, int W,
                const pl3d_params* p, const float* nd_host, int K, uint8_t* out_mask, float* out_normals,
                int32_t* out_labels, float* out_points, uint8_t* out_groups, const Tuning& t,
                int32_t* out_labels_copy) {
    memset(&a, 0, sizeof(a));
    a.points = points;
    a.H = H;
    a.W = W;
    a.lambda = p->lap_lambda;
    const bool tma_ok = (W % 4) == 0 && aligned16(points) && encode_fn() != nullptr;

    // Laplacian passes (Eq. 1-2): displacement ping-pong, the first pass reads no displacement.
    const int rl = p->lap_iters > 0 ? p->lap_kernel / 2 : 1;
    const int lfuse = fused_iters(p->lap_iters, kLapMaxHalo / rl, t.lap_fuse);
    int remaining = p->lap_iters;
    size_t smem = 0;
    do {
        if (a.n_lap == kMaxPasses) return PL3D_ERR_UNSUPPORTED;
        LapPhase& ph = a.lap[a.n_lap];
        ph.iters = remaining < lfuse ? remaining : lfuse;
        ph.halo = ph.iters * rl;
        const bool thin = lap_thin(ph.iters, a.n_lap == 0);
        ph.tile_h = lap_tile_h(ph.iters, a.n_lap == 0, ph.halo, t.lap_tile_h);
        ph.tiles = div_up(H, ph.tile_h) * div_up(W, kTile);
        ph.dbufs = thin ? 1 : 2;
        ph.box = lap_box(ph.halo, ph.tile_h);
        ph.use_tma = a.n_lap == 0 && tma_ok;
        ph.stages = ph.use_tma ? lap_stages_for(lap_box_floats(ph.halo, ph.tile_h), ph.dbufs) : 1;
        ph.d_in = a.n_lap == 0 ? nullptr : sc.disp[(a.n_lap - 1) & 1];
        ph.d_out = sc.disp[a.n_lap & 1];
        remaining -= ph.iters;
        ph.export_points = remaining == 0 ? out_points : nullptr;
        const size_t m = lap_smem_for(lap_box_floats(ph.halo, ph.tile_h), ph.stages, ph.dbufs);
        smem = m > smem ? m : smem;
        ++a.n_lap;
    } while (remaining > 0);
    a.disp = a.lap[a.n_lap - 1].d_out;
    if (a.lap[0].use_tma && !encode_aos(&a.tm_pts_lap, points, H, W, a.lap[0].box, true)) {
        a.lap[0].use_tma = 0;
        a.lap[0].stages = 1;
    }

    // Bilateral passes (Eq. 3-6) and the quads' finish (Algorithms 1, 4, 5).
    const int rb = p->bil_iters > 0 ? p->bil_kernel / 2 : 1;
    const int bfuse = fused_iters(p->bil_iters, kBilMaxHalo / rb, t.bil_fuse);
    const int nb = bilateral_passes(p, t);
    if (nb > kMaxPasses) return PL3D_ERR_UNSUPPORTED;
    const int bth = bil_tile_h(t);
    a.bil_th = bth;
    if (nb > 1 && (!sc.carry[0] || !sc.carry[1])) return PL3D_ERR_INVALID_ARG;
    int bremaining = p->bil_iters;
    for (int c = 0; c < nb; ++c) {
        BilPhase& ph = a.bil[c];
        ph.iters = bremaining < bfuse ? bremaining : bfuse;
        bremaining -= ph.iters;
        ph.halo = ph.iters * rb;
        ph.box = bil_box(ph.halo, bth);
        ph.first = c == 0;
        ph.last = c + 1 == nb;
        ph.carry_in = c > 0 ? sc.carry[(c - 1) & 1] : nullptr;
        ph.carry_out = c + 1 < nb ? sc.carry[c & 1] : nullptr;
        ph.use_tma = c == 0 && tma_ok && aligned16(a.disp);
        const size_t m = bil_smem(ph.halo, bth);
        smem = m > smem ? m : smem;
    }
    a.n_bil = nb;
    if (a.bil[0].use_tma && !(encode_aos(&a.tm_pts_bil, points, H, W, a.bil[0].box, true) &&
                              encode_aos(&a.tm_disp_bil, a.disp, H, W, a.bil[0].box, false)))
        a.bil[0].use_tma = 0;

    float c_scale = 1.f, a_norm = 0.f;
    bilateral_scales(p->bil_sigma_len, p->bil_sigma_ang, p->bil_iters, &c_scale, &a_norm);
    a.out_mask = out_mask;
    a.out_normals = out_normals;
    a.groups = out_groups ? out_groups : sc.groups;
    a.labels = out_labels;
    a.labels_copy = out_labels_copy;
    a.sizes = p->min_triangles > 0 ? sc.sizes : nullptr;
    a.c_scale = c_scale;
    a.a_norm = a_norm;
    a.max_edge2 = p->max_edge > 0.f ? p->max_edge * p->max_edge : INFINITY;
    a.min_dot = p->min_dot;
    a.max_offset = p->max_offset;
    a.max_offset_scaled = p->max_offset > 0.f ? p->max_offset * c_scale : 0.f;
    a.min_triangles = p->min_triangles;
    a.barrier = sc.barrier;
    a.error = sc.error;
    a.border = sc.border && sc.cap_border >= border_counters(H, W, t) ? sc.border : nullptr;
    a.phase_ns = sc.phase_ns;
    a.nd.K = K;
    for (int j = 0; j < K; ++j) {
        const double x = nd_host[3 * j], y = nd_host[3 * j + 1], z = nd_host[3 * j + 2];
        const double len = sqrt(x * x + y * y + z * z);
        a.nd.v[3 * j] = (float)(x / len);
        a.nd.v[3 * j + 1] = (float)(y / len);
        a.nd.v[3 * j + 2] = (float)(z / len);
    }

    plan.frame_fn = kernel_for(rl, rb);
    plan.batch_fn = batch_kernel_for(rl, rb);
    if (!plan.frame_fn || !plan.batch_fn) return PL3D_ERR_UNSUPPORTED;
    plan.rl = rl;
    plan.rb = rb;
    plan.smem = smem;
    plan.tiles_lap = 0;   // the most tiles of any Laplacian pass
    for (int c = 0; c < a.n_lap; ++c) plan.tiles_lap = std::max(plan.tiles_lap, a.lap[c].tiles);
    plan.tiles_bil = div_up(H - 1, bth) * div_up(W - 1, kTile);
    const int Hq = H - 1, Wq = W - 1;
    plan.merge_items = (long long)(div_up(Hq, bth) - 1) * Wq + (long long)(div_up(Wq, kTile) - 1) * Hq;
    plan.tris = 2LL * Hq * Wq;
    return PL3D_OK;
}

int persistent_grid(const void* fn, size_t smem, int dev, const Tuning& t, long long work) {
    int resident = resident_ctas(fn, smem, dev);
    if (resident <= 0) return 0;
    if (t.ctas_per_sm > 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        const long long want = (long long)t.ctas_per_sm * sms;
        if (want < resident) resident = (int)want;
    }
    return work < resident ? (int)(work > 0 ? work : 1) : resident;
}

bool lap1_eligible(const FrameArgs& a, int rl) {
    if (rl != 1) return false;
    for (int c = 0; c < a.n_lap; ++c)
        if (a.lap[c].iters > 1) return false;
    return true;
}

int lap1_grid(int dev, bool with_d, long long tasks) {
    const int resident = resident_ctas(lap1_kernel_for(with_d), lap1_smem_bytes(with_d), dev, kLap1Threads);
    if (resident <= 0 || tasks < 0) return resident;
    const long long need = (tasks + kLap1Threads / 32 - 1) / (kLap1Threads / 32);
    return need < resident ? (int)(need > 0 ? need : 1) : resident;
}

int frame_launch(const FrameScratch& sc, const float* points, int H, int W, const pl3d_params* p, const float* nd_host,
                 int K, uint8_t* out_mask, float* out_normals, int32_t* out_labels, float* out_points,
                 uint8_t* out_groups, const Tuning& t, cudaStream_t s, int32_t* out_labels_copy,
                 cudaEvent_t normals_ready, int* launches) {
    static_assert(sizeof(FrameArgs) < 32000, "kernel parameters must fit the 32 KB parameter space");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PL3D_ERR_CUDA;
    FrameArgs a;
    FramePlan plan;
    int rc = frame_build(a, plan, sc, points, H, W, p, nd_host, K, out_mask, out_normals, out_labels, out_points,
                         out_groups, t, out_labels_copy);
    if (rc != PL3D_OK) return rc;
    const int work = plan.tiles_lap > plan.tiles_bil ? plan.tiles_lap : plan.tiles_bil;
    const int grid = persistent_grid(plan.frame_fn, plan.smem, dev, t, work);
    if (grid <= 0) return PL3D_ERR_CUDA;
    int n_launched = 0;
    if (lap1_eligible(a, plan.rl)) {
        // the Laplacian passes as kernels of their own; the persistent kernel starts at the bilateral
        for (int c = 0; c < a.n_lap; ++c) {
            const LapPhase& ph = a.lap[c];
            Lap1Args la;
            memset(&la, 0, sizeof(la));
            la.one = Lap1Frame{points, ph.d_in, ph.d_out, ph.export_points, H, W, ph.iters, a.lambda};
            la.pass = c;
            la.stamp = sc.phase_ns ? sc.phase_ns + 4 : nullptr;
            la.phase_ns = sc.phase_ns;
            la.sched = sc.lap1_sched;
            const bool with_d = ph.d_in != nullptr;
            const int g = lap1_grid(dev, with_d, lap1_tasks(H, W));
            if (g <= 0) return PL3D_ERR_CUDA;
            void* largs[1] = {&la};
            if (cudaLaunchKernel(lap1_kernel_for(with_d), dim3(g), dim3(kLap1Threads), largs, lap1_smem_bytes(with_d),
                                 s) !=
                cudaSuccess) {
                cudaGetLastError();
                return PL3D_ERR_CUDA;
            }
            ++n_launched;
        }
        a.n_lap = 0;
    }
    // one launch, or two with the event between them: the first ends once mask, normals and
    // groups are final, the second joins the segments across tiles (the same arguments; the
    // merge phase joins the tile borders there, so that the first launch ends sooner)
    if (normals_ready) a.border = nullptr;
    void* args[1] = {&a};
    for (int part = normals_ready ? 1 : 0; part <= (normals_ready ? 2 : 0); ++part) {
        a.part = part;
        if (cudaLaunchCooperativeKernel(plan.frame_fn, dim3(grid), dim3(kThreads), args, plan.smem, s) != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_CUDA;
        }
        ++n_launched;
        if (part == 1 && cudaEventRecord(normals_ready, s) != cudaSuccess) return PL3D_ERR_CUDA;
    }
    if (launches) *launches = n_launched;
    return PL3D_OK;
}

}  // namespace pl3d

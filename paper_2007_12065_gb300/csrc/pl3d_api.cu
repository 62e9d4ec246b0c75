// pl3d_api.cu -- the C ABI declared in include/pl3d.h: argument checks, the context and its
// scratch memory, per-phase timing, the device error word, and the host-buffer entry point.
// The path itself is one cooperative launch of the frame kernel per call (frame_host.cu,
// frame_kernels.cuh): Laplacian passes, bilateral passes with the quads' finish and the
// tile-local segments, the segment merge across tiles, and the labels. Batches of frames
// (one launch for many frames) are in pl3d_batch.cu.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "pl3d_ctx.cuh"

using namespace pl3d;
using namespace pl3d::ctxutil;

namespace {

constexpr int kVersion = 2 * 10000 + 1 * 100 + 0;

const char* const kSlotNames[PL3D_TIMING_SLOTS] = {
    "laplacian",      "bilateral",     "label_merge",        "label_flatten",  "frame_kernel",
    "host_copies",    "mesh_kernel",   "fastga_kernel",      "bil_staging_cta", "bil_geometry_cta",
    "bil_iterations_cta", "bil_finish_cta", "bil_labels_cta"};
static_assert(kSlotBilStage0 + kBilStages == PL3D_TIMING_SLOTS, "timing slots");

bool finite_f(float x) { return isfinite(x) != 0; }

// groups and segment sizes share one capacity.
int grow_tri(pl3d_ctx* ctx, size_t need, cudaStream_t s) {
    if (ctx->cap_tri >= need) return PL3D_OK;
    if (ctx->groups && cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
    cudaFree(ctx->groups);
    cudaFree(ctx->sizes);
    ctx->groups = nullptr;
    ctx->sizes = nullptr;
    ctx->cap_tri = 0;
    const size_t n = need + need / 8;
    if (cudaMalloc((void**)&ctx->groups, n) != cudaSuccess ||
        cudaMalloc((void**)&ctx->sizes, n * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    ctx->cap_tri = n;
    return PL3D_OK;
}

// The tile-border counters start at zero (even: every launch adds two to each one it uses).
int grow_border(pl3d_ctx* ctx, size_t need, cudaStream_t s) {
    if (ctx->cap_border >= need) return PL3D_OK;
    int rc = grow(&ctx->border, &ctx->cap_border, need, 1, s);
    if (rc != PL3D_OK) return rc;
    return cudaMemsetAsync(ctx->border, 0, ctx->cap_border * sizeof(unsigned), s) == cudaSuccess ? PL3D_OK
                                                                                                : PL3D_ERR_CUDA;
}

// The device address of a page-locked (cudaHostAlloc'd or registered) host buffer, or nullptr
// for memory the device cannot address directly (pageable memory, device memory).
void* device_view(void* host) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int run(pl3d_ctx* ctx, const float* points, int H, int W, const pl3d_params* p, const float* nd_host, int K,
        uint8_t* out_mask, float* out_normals, int32_t* out_labels, float* out_points, uint8_t* out_groups,
        cudaStream_t s, int32_t* out_labels_copy = nullptr, cudaEvent_t normals_ready = nullptr) {
    const size_t npts = (size_t)H * W;
    const size_t ntri = 2 * (size_t)(H - 1) * (W - 1);
    int rc;
    if ((rc = grow(&ctx->disp, &ctx->cap_points, npts, 6, s)) != PL3D_OK) return rc;
    if ((rc = grow_tri(ctx, ntri, s)) != PL3D_OK) return rc;
    if ((rc = grow_border(ctx, border_counters(H, W, ctx->tuning), s)) != PL3D_OK) return rc;
    if (bilateral_passes(p, ctx->tuning) > 1 && (rc = grow(&ctx->carry, &ctx->cap_carry, ntri, 6, s)) != PL3D_OK) return rc;

    FrameScratch sc;
    sc.disp[0] = ctx->disp;
    sc.disp[1] = ctx->disp + 3 * ctx->cap_points;
    sc.carry[0] = ctx->carry;
    sc.carry[1] = ctx->carry ? ctx->carry + 3 * ctx->cap_carry : nullptr;
    sc.groups = ctx->groups;
    sc.sizes = ctx->sizes;
    sc.barrier = ctx->barrier();
    sc.error = ctx->error();
    sc.phase_ns = ctx->timing ? ctx->phase_ns() : nullptr;
    sc.lap1_sched = ctx->lap1_sched();
    sc.border = ctx->border;
    sc.cap_border = ctx->cap_border;
    sc.seed_flags = nullptr;
    sc.seed_centroids = nullptr;

    const bool seeded = (p->flags & PL3D_FLAG_SEED_PTP) != 0;
    pl3d_params q = *p;
    if (seeded) {
        // components first: no offset test, no tri_min (both belong to the seeded pass)
        if ((rc = grow(&ctx->seed_flags, &ctx->cap_seed, ntri, 1, s)) != PL3D_OK ||
            (rc = grow(&ctx->seed_centroids, &ctx->cap_seed_c, ntri, 3, s)) != PL3D_OK)
            return rc;
        sc.seed_flags = ctx->seed_flags;
        sc.seed_centroids = ctx->seed_centroids;
        q.max_offset = 0.f;
        q.min_triangles = 0;
        q.flags = 0;
    }
    cudaEvent_t e0, e1;
    record_start(ctx, s, &e0, &e1);
    int n_launched = 0;
    rc = frame_launch(sc, points, H, W, &q, nd_host, K, out_mask, out_normals, out_labels, out_points, out_groups,
                      ctx->tuning, s, seeded ? nullptr : out_labels_copy, normals_ready, &n_launched);
    record_stop(ctx, s, kSlotKernel, e0, e1);
    if (rc != PL3D_OK) return rc;
    if (seeded) {
        rc = seeded_labels(sc, final_disp(sc, &q, ctx->tuning), points, H, W, p, nd_host, K,
                           out_groups ? out_groups : ctx->groups, out_labels, s);
        if (rc != PL3D_OK) return rc;
        ctx->launches += 1;
    }
    ctx->launches += n_launched;
    if (ctx->timing) ctx->timed_frames += 1;
    return PL3D_OK;
}

}  // namespace

namespace pl3d {
namespace ctxutil {

int ctx_run(pl3d_ctx* ctx, const float* points, int H, int W, const pl3d_params* p, const float* nd_host, int K,
            uint8_t* out_mask, float* out_normals, int32_t* out_labels, cudaStream_t s) {
    return run(ctx, points, H, W, p, nd_host, K, out_mask, out_normals, out_labels, nullptr, nullptr, s);
}

int ctx_reserve(pl3d_ctx* ctx, size_t points, cudaStream_t s) {
    int rc = grow(&ctx->disp, &ctx->cap_points, points, 6, s);
    if (rc == PL3D_OK) rc = grow_tri(ctx, 2 * points, s);
    // tiles of 8 x 32 quads at the smallest height: at most about points / 16 of them, whatever
    // the frame's shape, and two counters each
    if (rc == PL3D_OK) rc = grow_border(ctx, points / 4 + 8, s);
    return rc;
}

}  // namespace ctxutil
}  // namespace pl3d

extern "C" {

int pl3d_version(void) { return kVersion; }

const char* pl3d_status_string(int status) {
    switch (status) {
        case PL3D_OK: return "ok";
        case PL3D_ERR_INVALID_ARG: return "invalid argument";
        case PL3D_ERR_OUT_OF_MEMORY: return "out of device memory";
        case PL3D_ERR_CUDA: return "CUDA error";
        case PL3D_ERR_TIMEOUT: return "device-side wait timed out";
        case PL3D_ERR_UNSUPPORTED: return "unsupported device or kernel size";
        default: return "unknown status";
    }
}

const char* pl3d_timing_slot_name(int slot) {
    if (slot < 0 || slot >= PL3D_TIMING_SLOTS) return "";
    return kSlotNames[slot];
}

int pl3d_default_params(pl3d_params* p) {
    if (!p) return PL3D_ERR_INVALID_ARG;
    p->lap_iters = 2;
    p->lap_lambda = 1.0f;
    p->lap_kernel = 3;
    p->bil_iters = 2;
    p->bil_sigma_len = 0.1f;
    p->bil_sigma_ang = 0.15f;
    p->bil_kernel = 3;
    p->max_edge = 0.05f;
    p->min_dot = 0.96f;
    p->max_offset = 0.0f;
    p->min_triangles = 0;
    p->flags = 0;
    return PL3D_OK;
}

int pl3d_validate(const pl3d_params* p, int H, int W, const float* nd, int K) {
    if (!p) return PL3D_ERR_INVALID_ARG;
    if (H < 2 || W < 2) return PL3D_ERR_INVALID_ARG;
    if (2LL * (H - 1) * (long long)(W - 1) >= (1LL << 31) || 3LL * H * W >= (1LL << 31)) return PL3D_ERR_INVALID_ARG;
    if (K < 1 || K > PL3D_MAX_GROUPS) return PL3D_ERR_INVALID_ARG;
    if ((p->flags & ~PL3D_FLAG_SEED_PTP) != 0) return PL3D_ERR_INVALID_ARG;
    if ((p->flags & PL3D_FLAG_SEED_PTP) && !(p->max_offset > 0.f)) return PL3D_ERR_INVALID_ARG;
    if (p->lap_iters < 0 || p->bil_iters < 0 || p->min_triangles < 0) return PL3D_ERR_INVALID_ARG;
    if (p->lap_iters > 0) {
        if (p->lap_kernel != 3 && p->lap_kernel != 5 && p->lap_kernel != 7) return PL3D_ERR_UNSUPPORTED;
        if (!finite_f(p->lap_lambda) || p->lap_lambda < 0.f || p->lap_lambda > 1.f) return PL3D_ERR_INVALID_ARG;
        if (p->lap_iters > kMaxPasses * (kLapMaxHalo / (p->lap_kernel / 2))) return PL3D_ERR_UNSUPPORTED;
    }
    if (p->bil_iters > 0) {
        if (p->bil_kernel != 3 && p->bil_kernel != 5 && p->bil_kernel != 7) return PL3D_ERR_UNSUPPORTED;
        if (!finite_f(p->bil_sigma_len) || !(p->bil_sigma_len > 0.f)) return PL3D_ERR_INVALID_ARG;
        if (!finite_f(p->bil_sigma_ang) || !(p->bil_sigma_ang > 0.f)) return PL3D_ERR_INVALID_ARG;
        if (p->bil_iters > kMaxPasses * (kBilMaxHalo / (p->bil_kernel / 2))) return PL3D_ERR_UNSUPPORTED;
    }
    if (!finite_f(p->max_edge) || !finite_f(p->min_dot) || !finite_f(p->max_offset)) return PL3D_ERR_INVALID_ARG;
    if (nd) {
        for (int j = 0; j < K; ++j) {
            const float x = nd[3 * j], y = nd[3 * j + 1], z = nd[3 * j + 2];
            if (!finite_f(x) || !finite_f(y) || !finite_f(z)) return PL3D_ERR_INVALID_ARG;
            if (x == 0.f && y == 0.f && z == 0.f) return PL3D_ERR_INVALID_ARG;
        }
    }
    return PL3D_OK;
}

int pl3d_create(pl3d_ctx** out, int cuda_device) {
    if (!out) return PL3D_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    if (cuda_device < 0 || cuda_device >= n) return PL3D_ERR_INVALID_ARG;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, cuda_device) != cudaSuccess) return PL3D_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return PL3D_ERR_UNSUPPORTED;
    if (!prop.cooperativeLaunch) return PL3D_ERR_UNSUPPORTED;
    DeviceGuard g(cuda_device);
    if (!g.ok) return PL3D_ERR_CUDA;
    if (frame_configure() != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    pl3d_ctx* c = new (std::nothrow) pl3d_ctx();
    if (!c) return PL3D_ERR_OUT_OF_MEMORY;
    c->device = cuda_device;
    if (cudaMalloc((void**)&c->ctl, kCtlBytes) != cudaSuccess || cudaMemset(c->ctl, 0, kCtlBytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->ctl);
        delete c;
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    *out = c;
    return PL3D_OK;
}

void pl3d_destroy(pl3d_ctx* c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        cudaDeviceSynchronize();
        cudaFree(c->disp);
        cudaFree(c->carry);
        cudaFree(c->groups);
        cudaFree(c->sizes);
        cudaFree(c->ctl);
        cudaFree(c->border);
        cudaFree(c->st_points);
        cudaFree(c->st_mask);
        cudaFree(c->st_normals);
        cudaFree(c->st_labels);
        if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
        if (c->normals_ready) cudaEventDestroy(c->normals_ready);
        if (c->normals_copied) cudaEventDestroy(c->normals_copied);
        drop_graphs(c);
        cudaFree(c->bslab);
        cudaFree(c->mslab);
        cudaFree(c->seed_flags);
        cudaFree(c->seed_centroids);
        cudaFree(c->ga_tables);
        cudaFree(c->bdesc);
        cudaFreeHost(c->bstage);
        if (c->bupload) cudaEventDestroy(c->bupload);
        for (auto& r : c->pending) {
            cudaEventDestroy(r.start);
            cudaEventDestroy(r.stop);
        }
        for (auto e : c->free_events) cudaEventDestroy(e);
        cudaGetLastError();
    }
    delete c;
}

int pl3d_extract_planes_ex(pl3d_ctx* ctx, const float* points, int H, int W, const pl3d_params* params,
                           const float* dominant_normals, int K, uint8_t* out_tri_mask, float* out_normals,
                           int32_t* out_labels, float* out_points, uint8_t* out_groups, void* stream) {
    if (!ctx || !points || !dominant_normals || !out_tri_mask || !out_normals || !out_labels)
        return PL3D_ERR_INVALID_ARG;
    int rc = pl3d_validate(params, H, W, dominant_normals, K);
    if (rc != PL3D_OK) return rc;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    return run(ctx, points, H, W, params, dominant_normals, K, out_tri_mask, out_normals, out_labels, out_points,
               out_groups, (cudaStream_t)stream);
}

int pl3d_extract_planes(pl3d_ctx* ctx, const float* points, int H, int W, const pl3d_params* params,
                        const float* dominant_normals, int K, uint8_t* out_tri_mask, float* out_normals,
                        int32_t* out_labels, void* stream) {
    return pl3d_extract_planes_ex(ctx, points, H, W, params, dominant_normals, K, out_tri_mask, out_normals,
                                  out_labels, nullptr, nullptr, stream);
}

int pl3d_extract_planes_host(pl3d_ctx* ctx, const float* host_points, int H, int W, const pl3d_params* params,
                             const float* dominant_normals, int K, uint8_t* host_tri_mask, float* host_normals,
                             int32_t* host_labels, void* stream) {
    if (!ctx || !host_points || !dominant_normals || !host_tri_mask || !host_normals || !host_labels)
        return PL3D_ERR_INVALID_ARG;
    int rc = pl3d_validate(params, H, W, dominant_normals, K);
    if (rc != PL3D_OK) return rc;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t npts = (size_t)H * W;
    const size_t ntri = 2 * (size_t)(H - 1) * (W - 1);
    if ((rc = grow(&ctx->st_points, &ctx->st_cap_points, npts, 3, s)) != PL3D_OK) return rc;
    if (ctx->st_cap_tri < ntri) {
        if (ctx->st_mask && cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
        cudaFree(ctx->st_mask);
        cudaFree(ctx->st_normals);
        cudaFree(ctx->st_labels);
        ctx->st_mask = nullptr;
        ctx->st_normals = nullptr;
        ctx->st_labels = nullptr;
        ctx->st_cap_tri = 0;
        const size_t n = ntri + ntri / 8;
        if (cudaMalloc((void**)&ctx->st_mask, n) != cudaSuccess ||
            cudaMalloc((void**)&ctx->st_normals, n * 3 * sizeof(float)) != cudaSuccess ||
            cudaMalloc((void**)&ctx->st_labels, n * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_OUT_OF_MEMORY;
        }
        ctx->st_cap_tri = n;
    }
    // A page-locked mask and labels buffer that the device can address is written by the kernel
    // itself: the mask as the tiles finish, the final labels by the last label phase (the labels
    // also serve as the union-find parents and stay in device memory). That spares two copies
    // after the kernel. The normals are copied: written from the tiles into host memory, their
    // 12-byte records would slow the kernel more than the copy costs.
    uint8_t* d_mask = static_cast<uint8_t*>(device_view(host_tri_mask));
    int32_t* d_labels = static_cast<int32_t*>(device_view(host_labels));
    const bool seeded = (params->flags & PL3D_FLAG_SEED_PTP) != 0;   // labels finished on the host
    if (seeded) d_labels = nullptr;
    // The normals are final before the segments across tiles: the path runs as two launches,
    // and the normals' copy runs on a second stream beside the second launch.
    // each created on first use and kept only once created; one that failed is tried again by
    // the next call
    auto make_event = [](cudaEvent_t* e) {
        cudaEvent_t t = nullptr;
        if (!*e && cudaEventCreateWithFlags(&t, cudaEventDisableTiming) == cudaSuccess) *e = t;
        return *e != nullptr;
    };
    if (!ctx->copy_stream) {
        cudaStream_t t = nullptr;
        if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) == cudaSuccess) ctx->copy_stream = t;
    }
    if (!ctx->copy_stream || !make_event(&ctx->normals_ready) || !make_event(&ctx->normals_copied)) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    cudaEvent_t e0, e1;
    record_start(ctx, s, &e0, &e1);
    if (cudaMemcpyAsync(ctx->st_points, host_points, npts * 3 * sizeof(float), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return PL3D_ERR_CUDA;
    record_stop(ctx, s, kSlotCopies, e0, e1);
    rc = run(ctx, ctx->st_points, H, W, params, dominant_normals, K, d_mask ? d_mask : ctx->st_mask, ctx->st_normals,
             ctx->st_labels, nullptr, nullptr, s, d_labels, ctx->normals_ready);
    if (rc != PL3D_OK) return rc;
    if (cudaStreamWaitEvent(ctx->copy_stream, ctx->normals_ready, 0) != cudaSuccess ||
        cudaMemcpyAsync(host_normals, ctx->st_normals, ntri * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                        ctx->copy_stream) != cudaSuccess ||
        cudaEventRecord(ctx->normals_copied, ctx->copy_stream) != cudaSuccess)
        return PL3D_ERR_CUDA;
    record_start(ctx, s, &e0, &e1);
    if ((!d_mask && cudaMemcpyAsync(host_tri_mask, ctx->st_mask, ntri, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        (!d_labels &&
         cudaMemcpyAsync(host_labels, ctx->st_labels, ntri * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaStreamWaitEvent(s, ctx->normals_copied, 0) != cudaSuccess)
        return PL3D_ERR_CUDA;
    record_stop(ctx, s, kSlotCopies, e0, e1);
    if (cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
    return PL3D_OK;
}

int pl3d_sync(pl3d_ctx* ctx, void* stream) {
    if (!ctx) return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PL3D_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return PL3D_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, ctx->error(), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PL3D_ERR_CUDA;
    if (err != 0) {
        // a wait gave up: results of the affected calls are void; reset the barrier state
        cudaMemset(ctx->ctl, 0, 4 * sizeof(unsigned));
        return PL3D_ERR_TIMEOUT;
    }
    return PL3D_OK;
}

int pl3d_set_timing(pl3d_ctx* ctx, int enable) {
    if (!ctx) return PL3D_ERR_INVALID_ARG;
    ctx->timing = enable != 0;
    return PL3D_OK;
}

int pl3d_read_timing(pl3d_ctx* ctx, double* ms_out, int64_t* launches_out, int n_slots, int reset) {
    if (!ctx || n_slots < 0) return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    for (auto& r : ctx->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.stop) != cudaSuccess) return PL3D_ERR_CUDA;
        if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
            ctx->slot_ms[r.slot] += ms;
            ctx->slot_n[r.slot] += 1;
        }
        ctx->free_events.push_back(r.start);
        ctx->free_events.push_back(r.stop);
    }
    ctx->pending.clear();
    if (cudaDeviceSynchronize() != cudaSuccess) return PL3D_ERR_CUDA;
    unsigned long long ns[kStageSlot + kBilStages];
    if (cudaMemcpy(ns, ctx->phase_ns(), sizeof(ns), cudaMemcpyDeviceToHost) != cudaSuccess) return PL3D_ERR_CUDA;
    double ms_all[PL3D_TIMING_SLOTS];
    int64_t n_all[PL3D_TIMING_SLOTS];
    for (int i = 0; i < PL3D_TIMING_SLOTS; ++i) {
        ms_all[i] = ctx->slot_ms[i];
        n_all[i] = ctx->slot_n[i];
    }
    for (int i = 0; i < 4; ++i) {
        ms_all[i] = (double)ns[i] * 1e-6;
        n_all[i] = ctx->timed_frames;
    }
    for (int i = 0; i < kBilStages; ++i) {
        ms_all[kSlotBilStage0 + i] = (double)ns[kStageSlot + i] * 1e-6;
        n_all[kSlotBilStage0 + i] = ctx->timed_frames;
    }
    for (int i = 0; i < n_slots && i < PL3D_TIMING_SLOTS; ++i) {
        if (ms_out) ms_out[i] = ms_all[i];
        if (launches_out) launches_out[i] = n_all[i];
    }
    if (reset) {
        for (int i = 0; i < PL3D_TIMING_SLOTS; ++i) {
            ctx->slot_ms[i] = 0.0;
            ctx->slot_n[i] = 0;
        }
        ctx->timed_frames = 0;
        // the phase totals and the stage totals (the lap1 stamps between them are zero at rest)
        if (cudaMemset(ctx->phase_ns(), 0, sizeof(ns)) != cudaSuccess) return PL3D_ERR_CUDA;
        if (cudaDeviceSynchronize() != cudaSuccess) return PL3D_ERR_CUDA;
    }
    return PL3D_TIMING_SLOTS;
}

int64_t pl3d_launch_count(const pl3d_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"

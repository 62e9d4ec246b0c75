// pl3d_pipeline.cu -- pipelined host-buffer frames (pl3d_pipeline_* in include/pl3d.h).
//
// A stream of frames from host memory through the single-frame path. Three CUDA streams carry
// the work: input copies, kernels, output copies. Frame i takes buffer set i % depth; its input
// copy waits for nothing but the copy engine, its kernels wait for its input copy, and its output
// copies wait for its kernels. So while frame i is in its kernels, frame i + 1's points come in
// and frame i - 1's results go out. The kernels share the context's scratch (displacements,
// groups, segment sizes, control words), which is safe because they run in submission order on
// the one kernel stream. A set is reused only after its previous frame has been waited for, on
// the host, so no copy ever overwrites buffers still in use.
//
// The context's device error word is copied out with each frame's outputs; a frame whose copy
// shows it set reports PL3D_ERR_TIMEOUT, and the word and the grid-barrier state are cleared
// once every stream has drained (as pl3d_sync does).
#include <string.h>

#include <new>
#include <vector>

#include "pl3d_ctx.cuh"

using namespace pl3d;
using namespace pl3d::ctxutil;

namespace {

constexpr int kMaxDepth = 16;
constexpr int kHistory = 1024;   // statuses kept for tickets already waited for

struct PipeSet {
    float* d_points = nullptr;
    uint8_t* d_mask = nullptr;
    float* d_normals = nullptr;
    int32_t* d_labels = nullptr;
    int* h_err = nullptr;              // page-locked copy of the error word after the frame
    cudaEvent_t in_done = nullptr;     // input copy finished
    cudaEvent_t k_done = nullptr;      // kernels finished
    cudaEvent_t out_done = nullptr;    // output copies finished
    uint64_t ticket = 0;               // frame in flight on this set, 0 = none
};

struct Kept {
    uint64_t ticket = 0;
    int status = PL3D_OK;
};

}  // namespace

struct pl3d_pipeline {
    int device = 0;
    pl3d_ctx* ctx = nullptr;
    size_t max_points = 0;
    int depth = 0;
    cudaStream_t s_in = nullptr, s_k = nullptr, s_out = nullptr;
    std::vector<PipeSet> sets;
    uint64_t next = 1;                 // ticket of the next frame
    std::vector<Kept> kept;            // [kHistory], by ticket % kHistory
};

namespace {

void free_sets(pl3d_pipeline* pl) {
    for (auto& s : pl->sets) {
        cudaFree(s.d_points);
        cudaFree(s.d_mask);
        cudaFree(s.d_normals);
        cudaFree(s.d_labels);
        cudaFreeHost(s.h_err);
        if (s.in_done) cudaEventDestroy(s.in_done);
        if (s.k_done) cudaEventDestroy(s.k_done);
        if (s.out_done) cudaEventDestroy(s.out_done);
    }
    pl->sets.clear();
}

void release(pl3d_pipeline* pl) {
    if (pl->s_in) cudaStreamSynchronize(pl->s_in);
    if (pl->s_k) cudaStreamSynchronize(pl->s_k);
    if (pl->s_out) cudaStreamSynchronize(pl->s_out);
    free_sets(pl);
    if (pl->s_in) cudaStreamDestroy(pl->s_in);
    if (pl->s_k) cudaStreamDestroy(pl->s_k);
    if (pl->s_out) cudaStreamDestroy(pl->s_out);
    if (pl->ctx) pl3d_destroy(pl->ctx);
    cudaGetLastError();
    delete pl;
}

int alloc_set(PipeSet& s, size_t points) {
    const size_t tri = 2 * points;   // 2(H-1)(W-1) < 2 H W
    if (cudaMalloc((void**)&s.d_points, points * 3 * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&s.d_mask, tri) != cudaSuccess ||
        cudaMalloc((void**)&s.d_normals, tri * 3 * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void**)&s.d_labels, tri * sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost((void**)&s.h_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    *s.h_err = 0;
    if (cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.k_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    return PL3D_OK;
}

// Waits for the frame on set `s` and returns its status; the set is free afterwards.
int finish(pl3d_pipeline* pl, PipeSet& s) {
    int status = PL3D_OK;
    if (cudaEventSynchronize(s.out_done) != cudaSuccess) {
        cudaGetLastError();
        status = PL3D_ERR_CUDA;
    } else if (*s.h_err != 0) {
        // a bounded wait gave up: drain everything, then clear the error word and the barrier
        status = PL3D_ERR_TIMEOUT;
        if (cudaStreamSynchronize(pl->s_in) != cudaSuccess || cudaStreamSynchronize(pl->s_k) != cudaSuccess ||
            cudaStreamSynchronize(pl->s_out) != cudaSuccess ||
            cudaMemset(pl->ctx->ctl, 0, 4 * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            status = PL3D_ERR_CUDA;
        }
    }
    Kept& k = pl->kept[s.ticket % kHistory];
    k.ticket = s.ticket;
    k.status = status;
    s.ticket = 0;
    *s.h_err = 0;
    return status;
}

}  // namespace

extern "C" {

int pl3d_pipeline_create(int device, int64_t max_points, int depth, pl3d_pipeline** out) {
    if (!out) return PL3D_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_points < 4 || depth < 1 || depth > kMaxDepth || 3 * max_points >= (1LL << 31))
        return PL3D_ERR_INVALID_ARG;
    pl3d_pipeline* pl = new (std::nothrow) pl3d_pipeline();
    if (!pl) return PL3D_ERR_OUT_OF_MEMORY;
    int rc = pl3d_create(&pl->ctx, device);
    if (rc != PL3D_OK) {
        delete pl;
        return rc;
    }
    DeviceGuard g(device);
    if (!g.ok) {
        release(pl);
        return PL3D_ERR_CUDA;
    }
    pl->device = device;
    pl->max_points = (size_t)max_points;
    pl->depth = depth;
    pl->kept.resize(kHistory);
    if (cudaStreamCreateWithFlags(&pl->s_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&pl->s_k, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&pl->s_out, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        release(pl);
        return PL3D_ERR_CUDA;
    }
    pl->sets.resize(depth);
    for (auto& s : pl->sets)
        if ((rc = alloc_set(s, pl->max_points)) != PL3D_OK) {
            release(pl);
            return rc;
        }
    if ((rc = ctx_reserve(pl->ctx, pl->max_points, pl->s_k)) != PL3D_OK) {
        release(pl);
        return rc;
    }
    *out = pl;
    return PL3D_OK;
}

int pl3d_pipeline_submit(pl3d_pipeline* pl, const float* host_points, int H, int W, const pl3d_params* params,
                         const float* dominant_normals, int K, uint8_t* host_tri_mask, float* host_normals,
                         int32_t* host_labels, uint64_t* ticket) {
    if (!pl || !host_points || !dominant_normals || !host_tri_mask || !host_normals || !host_labels || !ticket)
        return PL3D_ERR_INVALID_ARG;
    int rc = pl3d_validate(params, H, W, dominant_normals, K);
    if (rc != PL3D_OK) return rc;
    if (params->flags & PL3D_FLAG_SEED_PTP) return PL3D_ERR_UNSUPPORTED;
    const size_t npts = (size_t)H * W;
    const size_t ntri = 2 * (size_t)(H - 1) * (W - 1);
    if (npts > pl->max_points) return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(pl->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    const uint64_t t = pl->next;
    PipeSet& s = pl->sets[t % pl->depth];
    if (s.ticket != 0) finish(pl, s);   // its status is kept for a later wait
    // input copy; kernels after it; output copies (and the error word) after the kernels
    if (cudaMemcpyAsync(s.d_points, host_points, npts * 3 * sizeof(float), cudaMemcpyHostToDevice, pl->s_in) !=
            cudaSuccess ||
        cudaEventRecord(s.in_done, pl->s_in) != cudaSuccess || cudaStreamWaitEvent(pl->s_k, s.in_done, 0) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    rc = ctx_run(pl->ctx, s.d_points, H, W, params, dominant_normals, K, s.d_mask, s.d_normals, s.d_labels, pl->s_k);
    if (rc != PL3D_OK) return rc;
    if (cudaEventRecord(s.k_done, pl->s_k) != cudaSuccess || cudaStreamWaitEvent(pl->s_out, s.k_done, 0) != cudaSuccess ||
        cudaMemcpyAsync(host_tri_mask, s.d_mask, ntri, cudaMemcpyDeviceToHost, pl->s_out) != cudaSuccess ||
        cudaMemcpyAsync(host_normals, s.d_normals, ntri * 3 * sizeof(float), cudaMemcpyDeviceToHost, pl->s_out) !=
            cudaSuccess ||
        cudaMemcpyAsync(host_labels, s.d_labels, ntri * sizeof(int32_t), cudaMemcpyDeviceToHost, pl->s_out) !=
            cudaSuccess ||
        cudaMemcpyAsync(s.h_err, pl->ctx->error(), sizeof(int), cudaMemcpyDeviceToHost, pl->s_out) != cudaSuccess ||
        cudaEventRecord(s.out_done, pl->s_out) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    s.ticket = t;
    pl->next = t + 1;
    *ticket = t;
    return PL3D_OK;
}

int pl3d_pipeline_wait(pl3d_pipeline* pl, uint64_t ticket) {
    if (!pl || ticket == 0 || ticket >= pl->next) return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(pl->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    PipeSet& s = pl->sets[ticket % pl->depth];
    if (s.ticket == ticket) return finish(pl, s);
    const Kept& k = pl->kept[ticket % kHistory];
    return k.ticket == ticket ? k.status : PL3D_ERR_INVALID_ARG;
}

pl3d_ctx* pl3d_pipeline_context(pl3d_pipeline* pl) { return pl ? pl->ctx : nullptr; }

int pl3d_pipeline_destroy(pl3d_pipeline* pl) {
    if (!pl) return PL3D_OK;
    DeviceGuard g(pl->device);
    release(pl);
    return PL3D_OK;
}

}  // extern "C"

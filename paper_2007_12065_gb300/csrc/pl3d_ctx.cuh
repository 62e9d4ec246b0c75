// pl3d_ctx.cuh -- the context behind the C ABI (pl3d_api.cu, pl3d_batch.cu): scratch memory,
// the batch descriptor block and its graphs, launch-shape tuning, timing records.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "pl3d_internal.cuh"

namespace pl3d {
namespace ctxutil {

// Timing slots: four phases of the persistent kernels (device %globaltimer, accumulated by the
// kernel), the kernel as a whole, the host copies, the explicit-mesh launch and the Gaussian
// accumulator (CUDA events on the call's stream).
enum Slot { kSlotLap = 0, kSlotBil, kSlotMerge, kSlotLabels, kSlotKernel, kSlotCopies, kSlotMesh, kSlotFastga,
            kSlotBilStage0 };   // then the kBilStages bilateral stage totals (CTA time)

struct TimedRange {
    int slot;
    cudaEvent_t start, stop;
};

// One instantiated graph: n_l1 single-iteration Laplacian nodes, then the batch kernel as a
// cooperative kernel node. Their arguments point at the context's descriptor block, so the graph
// stays valid until that block moves.
struct BatchGraph {
    const void* fn;
    size_t smem;
    int grid;
    int n_l1;
    cudaGraphExec_t exec;
};

// barrier [2], error word, pad; phase totals [4]; lap1 timing stamps [3]; bilateral stage totals
// [5] (u64); lap1 task counter [2]
constexpr size_t kCtlBytes =
    4 * sizeof(unsigned) + (kStageSlot + kBilStages) * sizeof(unsigned long long) + 2 * sizeof(unsigned);

}  // namespace ctxutil
}  // namespace pl3d

struct pl3d_ctx {
    int device = 0;
    // scratch of the single-frame entry points (grown to the largest frame)
    float* disp = nullptr;          // 2 x 3 cap_points floats (AoS displacement ping-pong)
    size_t cap_points = 0;
    float* carry = nullptr;         // 2 x 3 cap_carry floats (multi-pass bilateral)
    size_t cap_carry = 0;
    uint8_t* groups = nullptr;      // cap_tri
    int32_t* sizes = nullptr;       // cap_tri
    size_t cap_tri = 0;
    unsigned* ctl = nullptr;        // control words (ctxutil::kCtlBytes): barrier, error, timing, lap1 counter
    unsigned* border = nullptr;     // cap_border tile-border counters of the single-frame kernel, even at rest
    size_t cap_border = 0;
    uint8_t* seed_flags = nullptr;  // PL3D_FLAG_SEED_PTP: per-root flags, cap_seed
    size_t cap_seed = 0;
    float* seed_centroids = nullptr;   // PL3D_FLAG_SEED_PTP: 3 cap_seed_c floats
    size_t cap_seed_c = 0;
    // device staging for the host-buffer entry point
    float* st_points = nullptr;
    size_t st_cap_points = 0;
    uint8_t* st_mask = nullptr;
    float* st_normals = nullptr;
    int32_t* st_labels = nullptr;
    size_t st_cap_tri = 0;
    // the host-buffer entry point copies the normals out on this stream while the second half
    // of the path (the segments across tiles) still runs on the caller's
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t normals_ready = nullptr;
    cudaEvent_t normals_copied = nullptr;
    // launch shape
    pl3d::Tuning tuning = {0, 0, 0};
    // batches: per-frame scratch slab, descriptor block (device + pinned staging), graphs
    unsigned char* bslab = nullptr;
    size_t bslab_cap = 0;
    unsigned char* bdesc = nullptr;
    unsigned char* bstage = nullptr;
    int bcap = 0;                   // frames the descriptor block holds
    std::vector<unsigned char> blast;   // bytes of the last upload
    cudaEvent_t bupload = nullptr;  // recorded after the last upload (staging may be rewritten after it)
    std::vector<pl3d::ctxutil::BatchGraph> graphs;
    int64_t graph_launches = 0;
    int64_t desc_uploads = 0;
    // scratch of the explicit-mesh launch (pl3d_mesh.cu)
    unsigned char* mslab = nullptr;
    size_t mslab_cap = 0;
    // Gaussian accumulator tables of one refinement level (pl3d_fastga.cu)
    unsigned char* ga_tables = nullptr;
    int ga_level = -1;
    size_t ga_smem_optin = 0;       // dynamic shared memory the accumulator kernel is opted in to
    size_t ga_off[3] = {0, 0, 0};
    // timing
    bool timing = false;
    int64_t timed_frames = 0;       // timed persistent launches
    std::vector<pl3d::ctxutil::TimedRange> pending;
    std::vector<cudaEvent_t> free_events;
    double slot_ms[PL3D_TIMING_SLOTS] = {};
    int64_t slot_n[PL3D_TIMING_SLOTS] = {};
    int64_t launches = 0;

    unsigned* barrier() const { return ctl; }
    int* error() const { return reinterpret_cast<int*>(ctl + 2); }
    unsigned long long* phase_ns() const { return reinterpret_cast<unsigned long long*>(ctl + 4); }
    unsigned* lap1_sched() const { return ctl + 4 + 2 * (pl3d::kStageSlot + pl3d::kBilStages); }
};

namespace pl3d {
namespace ctxutil {

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline cudaEvent_t take_event(pl3d_ctx* c) {
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

inline void record_start(pl3d_ctx* c, cudaStream_t s, cudaEvent_t* e0, cudaEvent_t* e1) {
    *e0 = *e1 = nullptr;
    if (!c->timing) return;
    *e0 = take_event(c);
    *e1 = take_event(c);
    if (*e0 && *e1) cudaEventRecord(*e0, s);
}

inline void record_stop(pl3d_ctx* c, cudaStream_t s, int slot, cudaEvent_t e0, cudaEvent_t e1) {
    if (!e0 || !e1) return;
    cudaEventRecord(e1, s);
    c->pending.push_back({slot, e0, e1});
}

// Frees and reallocates `*ptr` to hold `need` units of `elem_per` elements (plus headroom).
// Waits for the stream first, since work in flight may still use the old buffer.
template <class T>
int grow(T** ptr, size_t* cap, size_t need, size_t elem_per, cudaStream_t s) {
    if (*cap >= need) return PL3D_OK;
    if (*ptr) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
        cudaFree(*ptr);
        *ptr = nullptr;
        *cap = 0;
    }
    const size_t n = need + need / 8;
    if (cudaMalloc((void**)ptr, n * elem_per * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    *cap = n;
    return PL3D_OK;
}

// Drops the batch graphs (their arguments point into a descriptor block about to move).
void drop_graphs(pl3d_ctx* c);

// Slab bytes one frame of a batch takes under tuning t (pl3d_batch.cu).
size_t batch_scratch_bytes(const pl3d_frame& f, const Tuning& t);

// Grows the batch slab to `slab_bytes` and the descriptor block to `frames` frames now, so
// that later batches within those limits allocate nothing.
int batch_reserve(pl3d_ctx* c, size_t slab_bytes, int frames, cudaStream_t s);

// The single-frame path on device buffers, enqueued on `s` (pl3d_api.cu): the arguments checked
// as pl3d_extract_planes checks them; grows the context's scratch when a frame needs more.
int ctx_run(pl3d_ctx* ctx, const float* points, int H, int W, const pl3d_params* p, const float* nd_host, int K,
            uint8_t* out_mask, float* out_normals, int32_t* out_labels, cudaStream_t s);

// Sizes the context's scratch for frames of up to `points` points now (pl3d_api.cu).
int ctx_reserve(pl3d_ctx* ctx, size_t points, cudaStream_t s);

}  // namespace ctxutil
}  // namespace pl3d

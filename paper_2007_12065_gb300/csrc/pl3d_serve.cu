// pl3d_serve.cu -- a frame server with continuous batching (pl3d_server_*).
//
// One worker thread owns the slots. A slot is a stream, a context (batch scratch, descriptor
// block, graphs) and a device arena for the points and outputs of the requests it runs. The
// worker repeatedly (1) retires slots whose batch has finished -- a host function enqueued at
// the end of the batch's stream stamps the time and wakes the worker -- and (2) hands the
// waiting requests, oldest first, to a free slot: as many as the slot's arena and scratch have
// room for, up to max_batch_frames. Requests that arrive while a batch is on the GPU therefore
// join the next batch, which runs beside it on the other slot.
//
// Two batches in flight run side by side on the GPU (each is a cooperative kernel whose CTAs wait
// for one another): every slot of a two-slot server keeps its bilateral halo at 3 quads or less,
// so that each CTA fits half an SM's shared memory, and launches one CTA per SM while the other
// slot has a batch on the GPU. A slot that launches while the other one is idle takes two CTAs per
// SM, and a one-frame batch runs as a plain single-frame launch (no descriptor upload, no graph):
// at low arrival rates that is the sequential path's own launch. A grid launched while the other
// slot's grid fills the SMs waits for that grid's CTAs to finish; the other grid never waits for
// it, so nothing can deadlock.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "pl3d_ctx.cuh"

using namespace pl3d;
using namespace pl3d::ctxutil;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

constexpr size_t kAlign = 256;

struct Request {
    uint64_t ticket;
    const float* h_points;
    int H, W, K;
    pl3d_params params;
    std::vector<float> nd;
    uint8_t* h_mask;
    float* h_normals;
    int32_t* h_labels;
    int rl, rb;            // stencil radii the request constrains (0 = a filter that does not run)
    Tuning tuning;         // launch shape of a batch holding this request
    size_t arena_bytes;    // points + mask + normals + labels on the device
    size_t scratch_bytes;  // batch slab share
    int64_t t_submit;
    int64_t t_launch;
};

// Launch shape of a batch whose bilateral radius is rb. With two slots a batch that may run beside
// the other slot's takes one CTA per SM and a bilateral halo of at most 3 quads, so that a CTA
// takes at most half of an SM's shared memory; `alone` (the other slot idle) lifts the CTA limit.
Tuning slot_tuning(int max_inflight, int rb, bool alone = false) {
    if (max_inflight == 1) return Tuning{0, 0, 0};
    const int r = rb > 0 ? rb : 1;
    return Tuning{0, 3 / r > 0 ? 3 / r : 1, alone ? 0 : 1};
}

bool radii_match(int a, int b) { return a == 0 || b == 0 || a == b; }

size_t request_arena_bytes(int H, int W) {
    const size_t npts = (size_t)H * W, ntri = 2 * (size_t)(H - 1) * (W - 1);
    return align_up(npts * 12, kAlign) + align_up(ntri, kAlign) + align_up(ntri * 12, kAlign) +
           align_up(ntri * 4, kAlign);
}

}  // namespace

struct ServeSlot;

struct pl3d_server {
    pl3d_server_config cfg;
    std::vector<ServeSlot*> slots;
    std::thread worker;
    std::mutex mu;                        // pending, done, stop, counters below
    std::condition_variable wake;         // worker: a submission, a finished batch, stop
    std::condition_variable completed_cv; // pollers and drain
    std::deque<Request> pending;
    std::deque<pl3d_completion> done;
    bool stop = false;
    uint64_t next_ticket = 1;
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, triangles = 0;
    int64_t max_batch_seen = 0, max_inflight_seen = 0;
    int64_t outstanding = 0;              // submitted, not yet moved to `done`
    size_t arena_cap = 0, scratch_cap = 0;
    size_t slot_bytes = 0;
    int sms = 0;
};

struct ServeSlot {
    pl3d_server* srv = nullptr;
    pl3d_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    unsigned char* arena = nullptr;
    std::vector<Request> reqs;
    bool busy = false;
    std::atomic<int64_t> t_done{0};       // set by the stream's host function
    int status = PL3D_OK;
    int* h_err = nullptr;                 // page-locked copy of the context's device error word,
                                          // taken after each batch (before the host function)
};

namespace {

void CUDART_CB on_batch_done(void* user) {
    ServeSlot* s = static_cast<ServeSlot*>(user);
    s->t_done.store(now_ns(), std::memory_order_release);
    std::lock_guard<std::mutex> lock(s->srv->mu);
    s->srv->wake.notify_all();
}

// Enqueues the slot's requests: copies in, one batch (or one plain launch per frame), copies
// out, then the host function that marks the slot finished.
int launch_slot(pl3d_server* S, ServeSlot* sl) {
    std::vector<pl3d_frame> frames(sl->reqs.size());
    unsigned char* cur = sl->arena;
    int rc = PL3D_OK;
    for (size_t i = 0; i < sl->reqs.size() && rc == PL3D_OK; ++i) {
        Request& r = sl->reqs[i];
        const size_t npts = (size_t)r.H * r.W, ntri = 2 * (size_t)(r.H - 1) * (r.W - 1);
        pl3d_frame& f = frames[i];
        memset(&f, 0, sizeof(f));
        f.points = reinterpret_cast<float*>(cur);
        cur += align_up(npts * 12, kAlign);
        f.out_tri_mask = cur;
        cur += align_up(ntri, kAlign);
        f.out_normals = reinterpret_cast<float*>(cur);
        cur += align_up(ntri * 12, kAlign);
        f.out_labels = reinterpret_cast<int32_t*>(cur);
        cur += align_up(ntri * 4, kAlign);
        f.H = r.H;
        f.W = r.W;
        f.params = &r.params;
        f.dominant_normals = r.nd.data();
        f.K = r.K;
        if (cudaMemcpyAsync(const_cast<float*>(f.points), r.h_points, npts * 12, cudaMemcpyHostToDevice,
                            sl->stream) != cudaSuccess)
            rc = PL3D_ERR_CUDA;
    }
    if (rc == PL3D_OK) {
        if (S->cfg.max_batch_frames == 1 || frames.size() == 1) {
            for (size_t i = 0; i < frames.size() && rc == PL3D_OK; ++i) {
                const pl3d_frame& f = frames[i];
                rc = pl3d_extract_planes(sl->ctx, f.points, f.H, f.W, f.params, f.dominant_normals, f.K,
                                         f.out_tri_mask, f.out_normals, f.out_labels, sl->stream);
            }
        } else {
            rc = pl3d_extract_planes_batched(sl->ctx, frames.data(), (int)frames.size(), sl->stream);
        }
    }
    for (size_t i = 0; i < sl->reqs.size() && rc == PL3D_OK; ++i) {
        const Request& r = sl->reqs[i];
        const pl3d_frame& f = frames[i];
        const size_t ntri = 2 * (size_t)(r.H - 1) * (r.W - 1);
        if (cudaMemcpyAsync(r.h_mask, f.out_tri_mask, ntri, cudaMemcpyDeviceToHost, sl->stream) != cudaSuccess ||
            cudaMemcpyAsync(r.h_normals, f.out_normals, ntri * 12, cudaMemcpyDeviceToHost, sl->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(r.h_labels, f.out_labels, ntri * 4, cudaMemcpyDeviceToHost, sl->stream) != cudaSuccess)
            rc = PL3D_ERR_CUDA;
    }
    // the batch's device error word (a bounded wait that gave up) travels with the results
    if (rc == PL3D_OK && cudaMemcpyAsync(sl->h_err, sl->ctx->error(), sizeof(int), cudaMemcpyDeviceToHost,
                                         sl->stream) != cudaSuccess)
        rc = PL3D_ERR_CUDA;
    if (rc == PL3D_OK && cudaLaunchHostFunc(sl->stream, on_batch_done, sl) != cudaSuccess) rc = PL3D_ERR_CUDA;
    if (rc != PL3D_OK) {
        cudaGetLastError();
        cudaStreamSynchronize(sl->stream);   // nothing of this batch may still touch the buffers
        sl->t_done.store(now_ns(), std::memory_order_release);
    }
    return rc;
}

// Moves a finished slot's requests to the completion list (mu held). A batch whose device error
// word was set (a grid-barrier or TMA wait gave up) completes with PL3D_ERR_TIMEOUT, and the
// slot's control words start over before its next batch (ordered on the slot's stream).
void retire_slot(pl3d_server* S, ServeSlot* sl) {
    const int64_t t = sl->t_done.load(std::memory_order_acquire);
    if (sl->status == PL3D_OK && *sl->h_err != 0) {
        sl->status = PL3D_ERR_TIMEOUT;
        *sl->h_err = 0;
        if (cudaMemsetAsync(sl->ctx->ctl, 0, 4 * sizeof(unsigned), sl->stream) != cudaSuccess) cudaGetLastError();
    }
    for (const Request& r : sl->reqs) {
        pl3d_completion c;
        c.ticket = r.ticket;
        c.status = sl->status;
        c.batch_frames = (int32_t)sl->reqs.size();
        c.latency_ms = (double)(t - r.t_submit) * 1e-6;
        c.queue_ms = (double)(r.t_launch - r.t_submit) * 1e-6;
        S->done.push_back(c);
        S->completed += 1;
        S->outstanding -= 1;
        if (sl->status == PL3D_OK) S->triangles += 2LL * (r.H - 1) * (r.W - 1);
    }
    sl->reqs.clear();
    sl->busy = false;
    S->completed_cv.notify_all();
}

void worker_main(pl3d_server* S) {
    cudaSetDevice(S->cfg.device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        bool any_busy = false;
        for (ServeSlot* sl : S->slots) {
            if (sl->busy && sl->t_done.load(std::memory_order_acquire) != 0) retire_slot(S, sl);
            any_busy |= sl->busy;
        }
        if (S->stop && S->pending.empty() && !any_busy) break;
        // hand waiting requests to free slots, oldest first
        for (ServeSlot* sl : S->slots) {
            if (sl->busy || S->pending.empty()) continue;
            size_t arena = 0, scratch = 0;
            int rl = 0, rb = 0;
            while (!S->pending.empty() && (int)sl->reqs.size() < S->cfg.max_batch_frames) {
                const Request& r = S->pending.front();
                // one batch holds one Laplacian and one bilateral stencil size
                if (!radii_match(rl, r.rl) || !radii_match(rb, r.rb)) break;
                if (arena + r.arena_bytes > S->arena_cap || scratch + r.scratch_bytes > S->scratch_cap) break;
                arena += r.arena_bytes;
                scratch += r.scratch_bytes;
                rl = rl ? rl : r.rl;
                rb = rb ? rb : r.rb;
                sl->reqs.push_back(std::move(S->pending.front()));
                S->pending.pop_front();
            }
            if (sl->reqs.empty()) continue;
            bool alone = true;
            for (ServeSlot* o : S->slots) alone &= o == sl || !o->busy;
            sl->ctx->tuning = slot_tuning(S->cfg.max_inflight, rb, alone);
            sl->busy = true;
            sl->t_done.store(0, std::memory_order_relaxed);
            const int64_t t = now_ns();
            for (Request& r : sl->reqs) r.t_launch = t;
            S->batches += 1;
            S->max_batch_seen = std::max<int64_t>(S->max_batch_seen, (int64_t)sl->reqs.size());
            int inflight = 0;
            for (ServeSlot* o : S->slots) inflight += o->busy ? 1 : 0;
            S->max_inflight_seen = std::max<int64_t>(S->max_inflight_seen, inflight);
            lock.unlock();
            sl->status = launch_slot(S, sl);
            lock.lock();
        }
        bool finished = false;
        for (ServeSlot* sl : S->slots) finished |= sl->busy && sl->t_done.load(std::memory_order_acquire) != 0;
        if (finished) continue;
        bool can_launch = false;
        for (ServeSlot* sl : S->slots) can_launch |= !sl->busy;
        if (can_launch && !S->pending.empty()) continue;
        S->wake.wait_for(lock, std::chrono::milliseconds(5));
    }
}

void free_server(pl3d_server* S) {
    for (ServeSlot* sl : S->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        cudaFree(sl->arena);
        if (sl->h_err) cudaFreeHost(sl->h_err);
        if (sl->ctx) pl3d_destroy(sl->ctx);
        if (sl->stream) cudaStreamDestroy(sl->stream);
        delete sl;
    }
    S->slots.clear();
    cudaGetLastError();
}

}  // namespace

extern "C" {

int pl3d_server_create(pl3d_server** out, const pl3d_server_config* cfg) {
    if (!out) return PL3D_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg || cfg->max_inflight < 1 || cfg->max_inflight > 2 || cfg->max_batch_frames < 1 ||
        cfg->max_batch_frames > 4096 || cfg->reserved != 0 || cfg->hbm_bytes < 0)
        return PL3D_ERR_INVALID_ARG;
    pl3d_server* S = new (std::nothrow) pl3d_server();
    if (!S) return PL3D_ERR_OUT_OF_MEMORY;
    S->cfg = *cfg;
    DeviceGuard g(cfg->device);
    if (!g.ok) {
        delete S;
        return PL3D_ERR_INVALID_ARG;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return PL3D_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, cfg->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return PL3D_ERR_CUDA;
    }
    const size_t budget = cfg->hbm_bytes > 0 ? (size_t)cfg->hbm_bytes : free_b / 2;
    if (budget > free_b) {
        delete S;
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    // a slot's bytes split like one frame's needs: 46 B of buffers to 26 B of scratch per pixel
    const size_t per_slot = budget / cfg->max_inflight;
    S->arena_cap = per_slot / 72 * 46;
    S->scratch_cap = per_slot / 72 * 26 * 8 / 9;   // the slab allocator adds 1/8 of headroom
    int rc = PL3D_OK;
    for (int i = 0; i < cfg->max_inflight && rc == PL3D_OK; ++i) {
        ServeSlot* sl = new (std::nothrow) ServeSlot();
        if (!sl) {
            rc = PL3D_ERR_OUT_OF_MEMORY;
            break;
        }
        sl->srv = S;
        S->slots.push_back(sl);
        if ((rc = pl3d_create(&sl->ctx, cfg->device)) != PL3D_OK) break;
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) sl->stream = st;
        if (!sl->stream || cudaMalloc((void**)&sl->arena, S->arena_cap) != cudaSuccess ||
            cudaHostAlloc((void**)&sl->h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            rc = PL3D_ERR_OUT_OF_MEMORY;
            break;
        }
        *sl->h_err = 0;
        if (cfg->max_batch_frames > 1)
            rc = batch_reserve(sl->ctx, S->scratch_cap, cfg->max_batch_frames, sl->stream);
    }
    if (rc == PL3D_OK && cudaDeviceSynchronize() != cudaSuccess) rc = PL3D_ERR_CUDA;
    if (rc != PL3D_OK) {
        free_server(S);
        delete S;
        return rc;
    }
    S->slot_bytes = S->arena_cap + (S->slots[0]->ctx ? S->slots[0]->ctx->bslab_cap : 0);
    S->worker = std::thread(worker_main, S);
    *out = S;
    return PL3D_OK;
}

int pl3d_server_submit(pl3d_server* S, const float* host_points, int H, int W, const pl3d_params* params,
                       const float* nd, int K, uint8_t* host_tri_mask, float* host_normals, int32_t* host_labels,
                       uint64_t* ticket) {
    if (!S || !host_points || !params || !nd || !host_tri_mask || !host_normals || !host_labels)
        return PL3D_ERR_INVALID_ARG;
    int rc = pl3d_validate(params, H, W, nd, K);
    if (rc != PL3D_OK) return rc;
    if (params->flags & PL3D_FLAG_SEED_PTP) return PL3D_ERR_UNSUPPORTED;   // host-assisted: single frames
    Request r;
    r.h_points = host_points;
    r.H = H;
    r.W = W;
    r.K = K;
    r.params = *params;
    r.nd.assign(nd, nd + 3 * K);
    r.h_mask = host_tri_mask;
    r.h_normals = host_normals;
    r.h_labels = host_labels;
    r.rl = params->lap_iters > 0 ? params->lap_kernel / 2 : 0;
    r.rb = params->bil_iters > 0 ? params->bil_kernel / 2 : 0;
    r.tuning = slot_tuning(S->cfg.max_inflight, r.rb);
    r.arena_bytes = request_arena_bytes(H, W);
    pl3d_frame f;
    memset(&f, 0, sizeof(f));
    f.H = H;
    f.W = W;
    f.params = params;
    r.scratch_bytes = S->cfg.max_batch_frames > 1 ? batch_scratch_bytes(f, r.tuning) : 0;
    r.t_launch = 0;
    if (S->cfg.max_inflight > 1) {
        // both slots' kernels must fit on the GPU at once: two CTAs per SM for this frame
        const int rl = r.rl ? r.rl : 1, rb = r.rb ? r.rb : 1;
        const void* fn = batch_kernel_for_radii(rl, rb);
        DeviceGuard g(S->cfg.device);
        if (!fn || !g.ok || resident_ctas(fn, frame_smem_bytes(params, r.tuning), S->cfg.device) < 2 * S->sms)
            return PL3D_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) return PL3D_ERR_INVALID_ARG;
    if (r.arena_bytes > S->arena_cap || r.scratch_bytes > S->scratch_cap) {
        S->rejected += 1;
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    r.ticket = S->next_ticket++;
    r.t_submit = now_ns();
    if (ticket) *ticket = r.ticket;
    S->pending.push_back(std::move(r));
    S->submitted += 1;
    S->outstanding += 1;
    S->wake.notify_all();
    return PL3D_OK;
}

int pl3d_server_poll(pl3d_server* S, pl3d_completion* out, int max, int wait_ms) {
    if (!S || max < 0 || (max > 0 && !out)) return PL3D_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    if (S->done.empty() && wait_ms != 0) {
        auto ready = [&] { return !S->done.empty() || S->outstanding == 0; };
        if (wait_ms < 0) S->completed_cv.wait(lock, ready);
        else S->completed_cv.wait_for(lock, std::chrono::milliseconds(wait_ms), ready);
    }
    int n = 0;
    while (n < max && !S->done.empty()) {
        out[n++] = S->done.front();
        S->done.pop_front();
    }
    return n;
}

int pl3d_server_drain(pl3d_server* S) {
    if (!S) return PL3D_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    S->completed_cv.wait(lock, [&] { return S->outstanding == 0; });
    return PL3D_OK;
}

int pl3d_server_get_stats(const pl3d_server* S, pl3d_server_stats* out) {
    if (!S || !out) return PL3D_ERR_INVALID_ARG;
    pl3d_server* m = const_cast<pl3d_server*>(S);
    std::lock_guard<std::mutex> lock(m->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->batches = S->batches;
    out->triangles = S->triangles;
    out->max_batch_frames = S->max_batch_seen;
    out->max_inflight = S->max_inflight_seen;
    out->slot_bytes = (int64_t)S->slot_bytes;
    return PL3D_OK;
}

namespace {

// Linear-interpolation percentile of sorted values (q in [0, 1]).
double percentile_sorted(const std::vector<double>& v, double q) {
    if (v.empty()) return 0.0;
    const double pos = q * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = lo + 1 < v.size() ? lo + 1 : lo;
    return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

bool replay_args_ok(const pl3d_replay_source* src, int n_src, const double* arr, const int32_t* which, int64_t n) {
    for (int s = 0; s < n_src; ++s) {
        const pl3d_replay_source& r = src[s];
        if (!r.host_points || r.n_variants < 1 || r.ring < 1 || r.reserved != 0 || !r.params || !r.dominant_normals ||
            !r.host_mask || !r.host_normals || !r.host_labels)
            return false;
        for (int v = 0; v < r.n_variants; ++v)
            if (!r.host_points[v]) return false;
        for (int k = 0; k < r.ring; ++k)
            if (!r.host_mask[k] || !r.host_normals[k] || !r.host_labels[k]) return false;
    }
    double prev = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(arr[i] >= prev) || !std::isfinite(arr[i]) || which[i] < 0 || which[i] >= n_src) return false;
        prev = arr[i];
    }
    return true;
}

}  // namespace

int pl3d_server_replay(pl3d_server* S, const pl3d_replay_source* src, int n_src, const double* arr,
                       const int32_t* which, int64_t n, pl3d_replay_report* rep) {
    if (!S || !src || n_src < 1 || !arr || !which || n < 1 || !rep) return PL3D_ERR_INVALID_ARG;
    if (!replay_args_ok(src, n_src, arr, which, n)) return PL3D_ERR_INVALID_ARG;
    memset(rep, 0, sizeof(*rep));
    auto submit = [&](int s, int variant, int set, uint64_t* t) {
        const pl3d_replay_source& r = src[s];
        return pl3d_server_submit(S, r.host_points[variant], r.H, r.W, r.params, r.dominant_normals, r.K,
                                  r.host_mask[set], r.host_normals[set], r.host_labels[set], t);
    };
    std::vector<pl3d_completion> buf(1024);
    // warm-up: every frame of every source once, each on its own ring set in turn
    for (int s = 0; s < n_src; ++s)
        for (int v = 0; v < src[s].n_variants; ++v) {
            int rc = submit(s, v, v % src[s].ring, nullptr);
            if (rc == PL3D_OK && v % src[s].ring == src[s].ring - 1) rc = pl3d_server_drain(S);
            if (rc != PL3D_OK) return rc;
        }
    pl3d_server_drain(S);
    while (pl3d_server_poll(S, buf.data(), (int)buf.size(), 0) > 0) {
    }
    pl3d_server_stats st0;
    pl3d_server_get_stats(S, &st0);

    std::vector<int64_t> t_sched(n), t_call(n);
    std::vector<double> latency(n, 0.0);
    std::vector<int32_t> bframes(n, 0);
    std::vector<char> done(n, 0);
    std::vector<int32_t> status(n, PL3D_OK);
    std::vector<std::vector<int64_t>> owner(n_src);
    std::vector<int64_t> count(n_src, 0);
    for (int s = 0; s < n_src; ++s) owner[s].assign(src[s].ring, -1);
    uint64_t first = 0;
    int64_t n_done = 0;
    auto collect = [&](int wait_ms) {
        const int got = pl3d_server_poll(S, buf.data(), (int)buf.size(), wait_ms);
        if (got <= 0) return 0;
        for (int j = 0; j < got; ++j) {
            const pl3d_completion& c = buf[j];
            if (c.ticket < first || c.ticket - first >= (uint64_t)n) continue;
            const int64_t i = (int64_t)(c.ticket - first);
            done[i] = 1;
            status[i] = c.status;
            bframes[i] = c.batch_frames;
            // server latency runs from the submit call; add the time from the scheduled arrival
            latency[i] = c.latency_ms + (double)(t_call[i] - t_sched[i]) * 1e-6;
            ++n_done;
        }
        return got;
    };
    int rc = PL3D_OK;
    const int64_t t0 = now_ns();
    for (int64_t i = 0; i < n && rc == PL3D_OK; ++i) {
        t_sched[i] = t0 + (int64_t)(arr[i] * 1e9);
        for (;;) {
            const int64_t left = t_sched[i] - now_ns();
            if (left <= 0) break;
            if (left > 300000) {
                collect(0);
                const int64_t nap = std::min<int64_t>(left - 200000, 1000000);
                if (nap > 0) std::this_thread::sleep_for(std::chrono::nanoseconds(nap));
            }
        }
        const int s = which[i];
        const int64_t k = count[s]++;
        const int set = (int)(k % src[s].ring);
        const int64_t prev = owner[s][set];
        while (prev >= 0 && !done[prev]) collect(1);   // its output buffers are still in use
        t_call[i] = now_ns();
        uint64_t ticket = 0;
        rc = submit(s, (int)(k % src[s].n_variants), set, &ticket);
        if (rc != PL3D_OK) break;
        if (i == 0) first = ticket;
        owner[s][set] = i;
    }
    pl3d_server_drain(S);   // every submitted request has completed
    const int64_t t_end = now_ns();
    while (collect(0) > 0) {
    }
    if (rc != PL3D_OK) return rc;
    pl3d_server_stats st1;
    pl3d_server_get_stats(S, &st1);
    std::vector<double> lat;
    lat.reserve(n);
    double tris = 0.0, bsum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (!done[i]) continue;
        rep->completed += 1;
        if (status[i] != PL3D_OK) rep->failed += 1;
        lat.push_back(latency[i]);
        const pl3d_replay_source& r = src[which[i]];
        tris += 2.0 * (r.H - 1) * (double)(r.W - 1);
        bsum += bframes[i];
    }
    std::vector<double> lags(n);
    for (int64_t i = 0; i < n; ++i) lags[i] = (double)(t_call[i] - t_sched[i]) * 1e-6;
    std::sort(lat.begin(), lat.end());
    std::sort(lags.begin(), lags.end());
    const double wall = (double)(t_end - t0) * 1e-9;
    rep->requests = n;
    rep->batches = st1.batches - st0.batches;
    rep->max_batch_frames = st1.max_batch_frames;
    rep->max_inflight = st1.max_inflight;
    rep->seconds = wall;
    rep->p50_ms = percentile_sorted(lat, 0.50);
    rep->p90_ms = percentile_sorted(lat, 0.90);
    rep->p99_ms = percentile_sorted(lat, 0.99);
    rep->max_ms = lat.empty() ? 0.0 : lat.back();
    double sum = 0.0;
    for (double v : lat) sum += v;
    rep->mean_ms = lat.empty() ? 0.0 : sum / (double)lat.size();
    rep->mtri_s = wall > 0 ? tris / wall / 1e6 : 0.0;
    rep->achieved_fps = wall > 0 ? (double)rep->completed / wall : 0.0;
    rep->mean_batch_frames = rep->completed ? bsum / (double)rep->completed : 0.0;
    rep->submit_lag_p99_ms = percentile_sorted(lags, 0.99);
    return PL3D_OK;
}

void pl3d_server_destroy(pl3d_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->wake.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    {
        DeviceGuard g(S->cfg.device);
        free_server(S);
    }
    delete S;
}

}  // extern "C"

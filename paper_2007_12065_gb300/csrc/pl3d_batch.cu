// pl3d_batch.cu -- batches of frames in one persistent launch (pl3d_extract_planes_batched),
// the launch-shape tuning that every call uses, and the autotuner over it.
//
// A batch is described to the kernel by one device block (BatchHeader, per-pass prefix sums of
// the frames' tile counts, prefix sums of merge items and triangles, one FrameArgs per frame).
// The host fills the block in page-locked staging and copies it to the device only when it
// differs from the previous batch. The launch is a graph with one cooperative kernel node whose
// arguments point at the block, so one instantiated graph serves every batch of the same launch
// shape (kernel, shared memory, grid) until the block has to grow.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pl3d_ctx.cuh"

using namespace pl3d;
using namespace pl3d::ctxutil;

namespace pl3d {
namespace ctxutil {

void drop_graphs(pl3d_ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

}  // namespace ctxutil
}  // namespace pl3d

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte offsets of the descriptor block for `cap` frames.
struct DescLayout {
    size_t lap, bil, l1, merge, tris, frames, total;
    explicit DescLayout(int cap) {
        const size_t pre = (size_t)kMaxPasses * (cap + 1) * sizeof(int);
        lap = align_up(sizeof(BatchHeader), 128);
        bil = align_up(lap + pre, 128);
        l1 = align_up(bil + pre, 128);
        merge = align_up(l1 + pre, 128);
        tris = align_up(merge + (cap + 1) * sizeof(long long), 128);
        frames = align_up(tris + (cap + 1) * sizeof(long long), 128);
        total = frames + (size_t)cap * sizeof(FrameArgs);
    }
};
static_assert(sizeof(FrameArgs) % 64 == 0, "tensor maps in the descriptor block need 64-byte alignment");

// Scratch bytes one frame takes from the slab.
struct FrameNeeds {
    size_t disp, carry, groups, sizes;
    size_t total() const { return 2 * disp + 2 * carry + groups + sizes; }
};

FrameNeeds frame_needs(const pl3d_frame& f, const Tuning& t) {
    const size_t npts = (size_t)f.H * f.W;
    const size_t ntri = 2 * (size_t)(f.H - 1) * (f.W - 1);
    FrameNeeds n;
    n.disp = align_up(npts * 3 * sizeof(float), kAlign);
    n.carry = bilateral_passes(f.params, t) > 1 ? align_up(ntri * 3 * sizeof(float), kAlign) : 0;
    n.groups = f.out_groups ? 0 : align_up(ntri, kAlign);
    n.sizes = f.params->min_triangles > 0 ? align_up(ntri * sizeof(int32_t), kAlign) : 0;
    return n;
}

int grow_desc(pl3d_ctx* c, int n, cudaStream_t s) {
    if (c->bcap >= n) return PL3D_OK;
    if (c->bdesc && cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
    if (c->bupload && cudaEventSynchronize(c->bupload) != cudaSuccess) return PL3D_ERR_CUDA;
    drop_graphs(c);
    cudaFree(c->bdesc);
    cudaFreeHost(c->bstage);
    c->bdesc = nullptr;
    c->bstage = nullptr;
    c->bcap = 0;
    c->blast.clear();
    const int cap = n + n / 4 + 8;
    const DescLayout L(cap);
    if (cudaMalloc((void**)&c->bdesc, L.total) != cudaSuccess ||
        cudaMallocHost((void**)&c->bstage, L.total) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->bdesc);
        c->bdesc = nullptr;
        c->bstage = nullptr;
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    c->bcap = cap;
    return PL3D_OK;
}

int grow_slab(pl3d_ctx* c, size_t need, cudaStream_t s) {
    if (c->bslab_cap >= need) return PL3D_OK;
    if (c->bslab && cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
    cudaFree(c->bslab);
    c->bslab = nullptr;
    c->bslab_cap = 0;
    const size_t cap = need + need / 8;
    if (cudaMalloc((void**)&c->bslab, cap) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_OUT_OF_MEMORY;
    }
    c->bslab_cap = cap;
    return PL3D_OK;
}

// Graph for this launch shape: n_l1 single-iteration Laplacian passes (lap1_kernel, one node each,
// in pass order) and then the batch kernel as a cooperative node.
cudaGraphExec_t batch_graph(pl3d_ctx* c, const void* fn, size_t smem, int grid, const BatchArgs& args, int n_l1,
                            const Lap1Args* l1_args, const int* l1_grid) {
    for (auto& g : c->graphs)
        if (g.fn == fn && g.smem == smem && g.grid == grid && g.n_l1 == n_l1) return g.exec;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    bool ok = true;
    cudaGraphNode_t prev = nullptr;
    for (int i = 0; i < n_l1 && ok; ++i) {
        Lap1Args la = l1_args[i];
        void* lparams[1] = {&la};
        cudaKernelNodeParams lp;
        memset(&lp, 0, sizeof(lp));
        lp.func = const_cast<void*>(lap1_kernel_for(la.pass > 0));
        lp.gridDim = dim3(l1_grid[i]);
        lp.blockDim = dim3(kLap1Threads);
        lp.sharedMemBytes = (unsigned)lap1_smem_bytes(la.pass > 0);
        lp.kernelParams = lparams;
        cudaGraphNode_t node = nullptr;
        ok = cudaGraphAddKernelNode(&node, graph, prev ? &prev : nullptr, prev ? 1 : 0, &lp) == cudaSuccess;
        prev = node;
    }
    BatchArgs a = args;
    void* params[1] = {&a};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = const_cast<void*>(fn);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = params;
    cudaGraphNode_t node = nullptr;
    cudaLaunchAttributeValue coop;
    memset(&coop, 0, sizeof(coop));
    coop.cooperative = 1;
    ok = ok && cudaGraphAddKernelNode(&node, graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp) == cudaSuccess &&
         cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &coop) == cudaSuccess &&
         cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        return nullptr;
    }
    if (c->graphs.size() >= 16) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({fn, smem, grid, n_l1, exec});
    return exec;
}

int check_frames(const pl3d_frame* frames, int n, int* rl_out, int* rb_out) {
    int rl = 0, rb = 0;
    for (int i = 0; i < n; ++i) {
        const pl3d_frame& f = frames[i];
        if (!f.points || !f.params || !f.dominant_normals || !f.out_tri_mask || !f.out_normals || !f.out_labels)
            return PL3D_ERR_INVALID_ARG;
        const int rc = pl3d_validate(f.params, f.H, f.W, f.dominant_normals, f.K);
        if (rc != PL3D_OK) return rc;
        if (f.params->flags & PL3D_FLAG_SEED_PTP) return PL3D_ERR_UNSUPPORTED;   // host-assisted: single frames
        if (f.params->lap_iters > 0) {
            const int r = f.params->lap_kernel / 2;
            if (rl && r != rl) return PL3D_ERR_UNSUPPORTED;
            rl = r;
        }
        if (f.params->bil_iters > 0) {
            const int r = f.params->bil_kernel / 2;
            if (rb && r != rb) return PL3D_ERR_UNSUPPORTED;
            rb = r;
        }
    }
    *rl_out = rl ? rl : 1;
    *rb_out = rb ? rb : 1;
    return PL3D_OK;
}

int run_batch(pl3d_ctx* c, const pl3d_frame* frames, int n, cudaStream_t s) {
    int rl = 1, rb = 1;
    int rc = check_frames(frames, n, &rl, &rb);
    if (rc != PL3D_OK || n == 0) return rc;
    const Tuning t = c->tuning;

    size_t slab = 0;
    for (int i = 0; i < n; ++i) slab += frame_needs(frames[i], t).total();
    if ((rc = grow_slab(c, slab, s)) != PL3D_OK) return rc;
    if ((rc = grow_desc(c, n, s)) != PL3D_OK) return rc;
    // the staging block is rewritten below: the previous upload must have left it
    if (c->bupload && cudaEventSynchronize(c->bupload) != cudaSuccess) return PL3D_ERR_CUDA;

    const DescLayout L(c->bcap);
    const int stride = c->bcap + 1;
    unsigned char* st = c->bstage;
    BatchHeader* hdr = reinterpret_cast<BatchHeader*>(st);
    int* lap_pre = reinterpret_cast<int*>(st + L.lap);
    int* bil_pre = reinterpret_cast<int*>(st + L.bil);
    int* l1_pre = reinterpret_cast<int*>(st + L.l1);
    long long* merge_pre = reinterpret_cast<long long*>(st + L.merge);
    long long* tri_pre = reinterpret_cast<long long*>(st + L.tris);
    FrameArgs* fa = reinterpret_cast<FrameArgs*>(st + L.frames);
    memset(st, 0, L.frames);

    unsigned char* cursor = c->bslab;
    size_t smem = 0;
    int n_lap = 0, n_bil = 0, any_filter = 0;
    std::vector<int> bil_tiles(n), lap_passes(n), bil_passes(n);
    for (int i = 0; i < n; ++i) {
        const pl3d_frame& f = frames[i];
        const FrameNeeds need = frame_needs(f, t);
        FrameScratch sc;
        sc.disp[0] = reinterpret_cast<float*>(cursor);
        sc.disp[1] = reinterpret_cast<float*>(cursor + need.disp);
        cursor += 2 * need.disp;
        sc.carry[0] = need.carry ? reinterpret_cast<float*>(cursor) : nullptr;
        sc.carry[1] = need.carry ? reinterpret_cast<float*>(cursor + need.carry) : nullptr;
        cursor += 2 * need.carry;
        sc.groups = need.groups ? cursor : nullptr;
        cursor += need.groups;
        sc.sizes = need.sizes ? reinterpret_cast<int32_t*>(cursor) : nullptr;
        cursor += need.sizes;
        sc.barrier = c->barrier();
        sc.error = c->error();
        sc.phase_ns = nullptr;
        sc.lap1_sched = c->lap1_sched();
        sc.border = nullptr;   // the batch kernel joins the tile borders in its merge phase
        sc.cap_border = 0;
        FramePlan plan;
        rc = frame_build(fa[i], plan, sc, f.points, f.H, f.W, f.params, f.dominant_normals, f.K, f.out_tri_mask,
                         f.out_normals, f.out_labels, f.out_points, f.out_groups, t);
        if (rc != PL3D_OK) return rc;
        smem = std::max(smem, plan.smem);
        bil_tiles[i] = plan.tiles_bil;
        lap_passes[i] = fa[i].n_lap;
        bil_passes[i] = fa[i].n_bil;
        n_lap = std::max(n_lap, fa[i].n_lap);
        n_bil = std::max(n_bil, fa[i].n_bil);
        if (f.params->min_triangles > 0) any_filter = 1;
        merge_pre[i + 1] = merge_pre[i] + plan.merge_items;
        tri_pre[i + 1] = tri_pre[i] + plan.tris;
    }
    // every frame's Laplacian passes single-iteration with a 3 x 3 window: they run as lap1_kernel
    // nodes of the graph, and the batch kernel starts at the bilateral
    bool thin = rl == 1;
    for (int i = 0; i < n && thin; ++i) thin = lap1_eligible(fa[i], 1);
    const int n_l1 = thin ? n_lap : 0;
    long long most_tiles = 0;
    for (int pass = 0; pass < kMaxPasses; ++pass) {
        int* lp = lap_pre + pass * stride;
        int* bp = bil_pre + pass * stride;
        int* l1p = l1_pre + pass * stride;
        for (int i = 0; i < n; ++i) {
            lp[i + 1] = lp[i] + (pass < lap_passes[i] && !thin ? fa[i].lap[pass].tiles : 0);
            bp[i + 1] = bp[i] + (pass < bil_passes[i] ? bil_tiles[i] : 0);
            l1p[i + 1] = l1p[i] + (pass < lap_passes[i] && thin ? lap1_tasks(fa[i].H, fa[i].W) : 0);
        }
        most_tiles = std::max(most_tiles, (long long)std::max(lp[n], bp[n]));
    }
    if (thin) n_lap = 0;
    // per Laplacian pass: buffers sized for the largest box; staged ahead when some frame stages
    // by TMA, as many boxes as still fit two CTAs per SM
    for (int lp_pass = 0; lp_pass < n_lap; ++lp_pass) {
        int P = 0, dbufs = 1;
        bool tma = false;
        for (int i = 0; i < n; ++i) {
            if (lp_pass >= fa[i].n_lap) continue;
            const LapPhase& ph = fa[i].lap[lp_pass];
            P = std::max(P, lap_box_floats(ph.halo, ph.tile_h));
            dbufs = std::max(dbufs, ph.dbufs);
            tma |= ph.use_tma != 0;
        }
        const int ns = tma ? lap_stages_for(P, dbufs) : 1;
        hdr->lap_buf[lp_pass] = P;
        hdr->lap_stages[lp_pass] = ns;
        hdr->lap_dbufs[lp_pass] = dbufs;
        smem = std::max(smem, lap_smem_for(P, ns, dbufs));
    }
    hdr->n = n;
    hdr->n_lap = n_lap;
    hdr->n_bil = n_bil;
    hdr->any_filter = any_filter;
    hdr->timing = c->timing ? 1 : 0;

    // upload unless the device already holds exactly these bytes
    const size_t used = L.frames + (size_t)n * sizeof(FrameArgs);
    if (c->blast.size() != used || memcmp(c->blast.data(), st, used) != 0) {
        if (cudaMemcpyAsync(c->bdesc, st, used, cudaMemcpyHostToDevice, s) != cudaSuccess) return PL3D_ERR_CUDA;
        if (!c->bupload) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return PL3D_ERR_CUDA;
            }
            c->bupload = e;
        }
        if (cudaEventRecord(c->bupload, s) != cudaSuccess) return PL3D_ERR_CUDA;
        c->blast.assign(st, st + used);
        c->desc_uploads += 1;
    }

    BatchArgs args;
    args.hdr = reinterpret_cast<const BatchHeader*>(c->bdesc);
    args.lap_tiles = reinterpret_cast<const int*>(c->bdesc + L.lap);
    args.bil_tiles = reinterpret_cast<const int*>(c->bdesc + L.bil);
    args.merge_items = reinterpret_cast<const long long*>(c->bdesc + L.merge);
    args.tris = reinterpret_cast<const long long*>(c->bdesc + L.tris);
    args.frames = reinterpret_cast<const FrameArgs*>(c->bdesc + L.frames);
    args.stride = stride;
    args.barrier = c->barrier();
    args.error = c->error();
    args.phase_ns = c->phase_ns();

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PL3D_ERR_CUDA;
    const void* fn = batch_kernel_for_radii(rl, rb);
    if (!fn) return PL3D_ERR_UNSUPPORTED;
    const int grid = persistent_grid(fn, smem, dev, t, most_tiles);
    if (grid <= 0) return PL3D_ERR_CUDA;

    Lap1Args l1_args[kMaxPasses];
    int l1_grid[kMaxPasses];
    for (int pass = 0; pass < n_l1; ++pass) {
        Lap1Args& la = l1_args[pass];
        memset(&la, 0, sizeof(la));
        la.hdr = args.hdr;
        la.frames = args.frames;
        la.task_pre = reinterpret_cast<const int*>(c->bdesc + L.l1) + pass * stride;
        la.pass = pass;
        la.stamp = c->phase_ns() + 4;
        la.phase_ns = c->phase_ns();
        la.sched = c->lap1_sched();
        l1_grid[pass] = lap1_grid(dev, pass > 0, -1);
        if (l1_grid[pass] <= 0) return PL3D_ERR_CUDA;
    }

    cudaEvent_t e0, e1;
    record_start(c, s, &e0, &e1);
    cudaGraphExec_t exec = batch_graph(c, fn, smem, grid, args, n_l1, l1_args, l1_grid);
    if (!exec) return PL3D_ERR_CUDA;
    if (cudaGraphLaunch(exec, s) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    record_stop(c, s, kSlotKernel, e0, e1);
    c->graph_launches += 1;
    c->launches += 1 + n_l1;
    if (c->timing) c->timed_frames += 1;
    return PL3D_OK;
}

bool tuning_ok(const pl3d_tuning* t) {
    const bool lap_h = t->lap_tile_h == 0 ||
                       (t->lap_tile_h % 8 == 0 && t->lap_tile_h >= kLapMinTileH && t->lap_tile_h <= kLapMaxTileH);
    const bool bil_h = t->bil_tile_h == 0 ||
                       (t->bil_tile_h % 8 == 0 && t->bil_tile_h >= kBilMinTileH && t->bil_tile_h <= kBilMaxTileH);
    return t->lap_fuse >= 0 && t->bil_fuse >= 0 && t->ctas_per_sm >= 0 && lap_h && bil_h;
}

// Fused depths worth trying for `iters` iterations of a filter whose halo allows `max_fuse`:
// everything in as few passes as possible, then two and three passes, and with `single` one
// iteration per pass (the Laplacian with a 3 x 3 window, which then runs as lap1_kernel).
std::vector<int> fuse_candidates(int iters, int max_fuse, bool single = false) {
    std::vector<int> v;
    if (single && iters > 1 && iters <= kMaxPasses) v.push_back(1);
    for (int passes = 1; passes <= 3; ++passes) {
        int f = (iters + passes - 1) / passes;
        if (f > max_fuse) continue;
        if (f < 1) f = 1;
        if (std::find(v.begin(), v.end(), f) == v.end()) v.push_back(f);
    }
    if (v.empty()) v.push_back(0);
    return v;
}

}  // namespace

namespace pl3d {
namespace ctxutil {

size_t batch_scratch_bytes(const pl3d_frame& f, const Tuning& t) { return frame_needs(f, t).total(); }

int batch_reserve(pl3d_ctx* c, size_t slab_bytes, int frames, cudaStream_t s) {
    int rc = grow_slab(c, slab_bytes, s);
    if (rc == PL3D_OK) rc = grow_desc(c, frames, s);
    return rc;
}

}  // namespace ctxutil
}  // namespace pl3d

extern "C" {

int pl3d_extract_planes_batched(pl3d_ctx* ctx, const pl3d_frame* frames, int n, void* stream) {
    if (!ctx || n < 0 || (n > 0 && !frames)) return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    return run_batch(ctx, frames, n, (cudaStream_t)stream);
}

int pl3d_set_tuning(pl3d_ctx* ctx, const pl3d_tuning* t) {
    if (!ctx) return PL3D_ERR_INVALID_ARG;
    if (!t) {
        ctx->tuning = Tuning{0, 0, 0, 0, 0};
        return PL3D_OK;
    }
    if (!tuning_ok(t)) return PL3D_ERR_INVALID_ARG;
    ctx->tuning = Tuning{t->lap_fuse, t->bil_fuse, t->ctas_per_sm, t->lap_tile_h, t->bil_tile_h};
    return PL3D_OK;
}

int pl3d_get_tuning(const pl3d_ctx* ctx, pl3d_tuning* t) {
    if (!ctx || !t) return PL3D_ERR_INVALID_ARG;
    t->lap_fuse = ctx->tuning.lap_fuse;
    t->bil_fuse = ctx->tuning.bil_fuse;
    t->ctas_per_sm = ctx->tuning.ctas_per_sm;
    t->lap_tile_h = ctx->tuning.lap_tile_h;
    t->bil_tile_h = ctx->tuning.bil_tile_h;
    return PL3D_OK;
}

int pl3d_autotune_batched(pl3d_ctx* ctx, const pl3d_frame* frames, int n, void* stream, int reps,
                          pl3d_tuning* best, double* best_ms) {
    if (!ctx || n < 1 || !frames || reps < 1 || reps > 50) return PL3D_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int rl = 1, rb = 1;
    int rc = check_frames(frames, n, &rl, &rb);
    if (rc != PL3D_OK) return rc;
    int lap_iters = 0, bil_iters = 0;
    for (int i = 0; i < n; ++i) {
        lap_iters = std::max(lap_iters, (int)frames[i].params->lap_iters);
        bil_iters = std::max(bil_iters, (int)frames[i].params->bil_iters);
    }
    std::vector<Tuning> round1;
    for (int lf : fuse_candidates(lap_iters, kLapMaxHalo / rl, rl == 1))
        for (int bf : fuse_candidates(bil_iters, kBilMaxHalo / rb))
            for (int cps : {1, 2}) round1.push_back(Tuning{lf, bf, cps, 0, 0});

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return PL3D_ERR_CUDA;
    }
    const Tuning saved = ctx->tuning;
    const bool saved_timing = ctx->timing;
    ctx->timing = false;
    double best_t = INFINITY;
    Tuning best_c = saved;
    std::vector<double> times;
    auto try_all = [&](const std::vector<Tuning>& cands) {
        for (const Tuning& cand : cands) {
            ctx->tuning = cand;
            if ((rc = run_batch(ctx, frames, n, s)) != PL3D_OK) return;
            times.clear();
            for (int r = 0; r < reps && rc == PL3D_OK; ++r) {
                float ms = 0.f;
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = PL3D_ERR_CUDA;
                if (rc == PL3D_OK) rc = run_batch(ctx, frames, n, s);
                if (rc == PL3D_OK && (cudaEventRecord(e1, s) != cudaSuccess ||
                                      cudaEventSynchronize(e1) != cudaSuccess ||
                                      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    rc = PL3D_ERR_CUDA;
                times.push_back(ms);
            }
            if (rc != PL3D_OK) return;
            std::sort(times.begin(), times.end());
            const double med = times[times.size() / 2];
            if (med < best_t) {
                best_t = med;
                best_c = cand;
            }
        }
    };
    // stage 1: fused depths and CTAs per SM at the default tile shapes; stage 2: tile heights at
    // the best of those (the default shape is stage 1's own entry)
    try_all(round1);
    if (rc == PL3D_OK) {
        std::vector<Tuning> round2;
        for (int lh : {16, 32, 48, 64})
            for (int bh : {16, 24, 32}) {
                Tuning c = best_c;
                c.lap_tile_h = lh;
                c.bil_tile_h = bh == kTile ? 0 : bh;
                if (c.lap_tile_h == kTile) c.lap_tile_h = 0;
                if (c.lap_tile_h != 0 || c.bil_tile_h != 0) round2.push_back(c);
            }
        try_all(round2);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = saved_timing;
    if (rc != PL3D_OK) {
        ctx->tuning = saved;
        cudaGetLastError();
        return rc;
    }
    ctx->tuning = best_c;
    if ((rc = run_batch(ctx, frames, n, s)) != PL3D_OK) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PL3D_ERR_CUDA;
    if (best) {
        best->lap_fuse = best_c.lap_fuse;
        best->bil_fuse = best_c.bil_fuse;
        best->ctas_per_sm = best_c.ctas_per_sm;
        best->lap_tile_h = best_c.lap_tile_h;
        best->bil_tile_h = best_c.bil_tile_h;
    }
    if (best_ms) *best_ms = best_t;
    return PL3D_OK;
}

int pl3d_batch_stats(const pl3d_ctx* ctx, int64_t* graph_launches, int64_t* desc_uploads, int64_t* graphs) {
    if (!ctx) return PL3D_ERR_INVALID_ARG;
    if (graph_launches) *graph_launches = ctx->graph_launches;
    if (desc_uploads) *desc_uploads = ctx->desc_uploads;
    if (graphs) *graphs = (int64_t)ctx->graphs.size();
    return PL3D_OK;
}

}  // extern "C"

/*
 * pl3d.h -- C ABI of the GB300 (sm_103a) plane-extraction path for organized point
 * clouds, after Polylidar3D (Castagno & Atkins, arXiv 2007.12065).
 *
 * One call runs, on the caller's CUDA stream and entirely in this library's kernels:
 *
 *   1. Laplacian vertex smoothing on the implicit image grid       (Eq. 1-2, Section 5.1)
 *   2. centroids and unit normals of every triangle of T_FC        (Section 4.2, Section 5.2)
 *   3. bilateral filtering of the triangle normals                 (Eq. 3-6, Section 5.2)
 *   4. triangle mask: all vertices valid and longest edge <= l_max (Algorithm 1, Algorithm 4)
 *   5. group assignment against the K dominant normals             (Algorithm 4)
 *   6. connected planar segments of equal group over twin edges    (Algorithm 5, Algorithm 2)
 *
 * Mesh conventions (Section 4.2, Algorithm 1). The cloud is an H x W grid (the paper's
 * M x N) of FP32 xyz points, row-major, 12 bytes per point; a point with any non-finite
 * coordinate is invalid. Coordinates must stay below 1e18 in magnitude (squared distances
 * are formed in FP32); a point beyond that is treated as invalid too. Quad (u, v), 0 <= u < H-1, 0 <= v < W-1, has the points
 * p1 = (u, v), p2 = (u, v+1), p3 = (u+1, v+1), p4 = (u+1, v) and two triangles,
 * first = {p3, p2, p1} (k = 0) and second = {p1, p4, p3} (k = 1). Every per-triangle array
 * has 2 (H-1)(W-1) entries indexed by GID = 2 (u (W-1) + v) + k. Normals follow the
 * right-hand rule over that vertex order.
 *
 * Errors: every entry point returns PL3D_OK (0) or a negative PL3D_ERR_* code and never
 * aborts the process. Invalid arguments are rejected on the host before anything is
 * enqueued. Launches are asynchronous: a fault inside a kernel surfaces as
 * PL3D_ERR_CUDA from a later call or from pl3d_sync.
 *
 * Threading: a context is used by one host thread at a time. Calls on one context are
 * ordered on the stream they are given; calls on different streams with one context
 * must not overlap because they share the context's scratch memory.
 */
#ifndef PL3D_H
#define PL3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PL3D_OK 0
#define PL3D_ERR_INVALID_ARG (-1)   /* null pointer, bad size, bad parameter */
#define PL3D_ERR_OUT_OF_MEMORY (-2) /* scratch or staging allocation failed */
#define PL3D_ERR_CUDA (-3)          /* a CUDA runtime call or a launch failed */
#define PL3D_ERR_TIMEOUT (-4)       /* a bounded device-side wait gave up */
#define PL3D_ERR_UNSUPPORTED (-5)   /* device is not sm_103-class, or an unsupported kernel size */

/* Largest number of dominant normals: groups are uint8 with 255 = "no group" (Algorithm 4). */
#define PL3D_MAX_GROUPS 254
/* Group value of a triangle that belongs to no dominant normal. */
#define PL3D_NO_GROUP 255

typedef struct pl3d_ctx pl3d_ctx;

/*
 * Parameters of one extraction. Paper symbols in brackets.
 *   lap_iters      Laplacian iterations (>= 0). Eq. 1.
 *   lap_lambda     [lambda] step in [0, 1]. Eq. 1, used as v' = v + lambda/W sum_j w_j (v_j - v),
 *                  w_j = 1 / |v - v_j| over the valid points of the lap_kernel x lap_kernel window
 *                  (the point itself and points at distance 0 excluded); the ring of width
 *                  lap_kernel/2 at the image border is not filtered (Section 5.1).
 *   lap_kernel     window size: 3, 5 or 7.
 *   bil_iters      bilateral iterations (>= 0). Eq. 3.
 *   bil_sigma_len  [sigma_c] metres, > 0: W_c = exp(-|c_i - c_j|^2 / (2 sigma_c^2)). Eq. 4.
 *   bil_sigma_ang  [sigma_s] > 0: W_s = exp(-|n_i - n_j|^2 / (2 sigma_s^2)). Eq. 5.
 *   bil_kernel     quad window size: 3, 5 or 7. The window of a triangle is both triangles of
 *                  every quad of the bil_kernel x bil_kernel quad block centred on its own quad,
 *                  itself included; triangles without a normal are skipped; the weighted sum is
 *                  renormalised to unit length each iteration; centroids stay fixed.
 *   max_edge       [l_max] metres; a triangle whose longest smoothed edge is > max_edge is
 *                  rejected. <= 0 disables the test. Algorithm 4.
 *   min_dot        [ang_min] a triangle joins group argmax_j n . n^d_j (lowest j on ties) unless
 *                  that dot is < min_dot. Algorithm 4.
 *   max_offset     if > 0, two adjacent triangles of group g join only when
 *                  |n^d_g . (c_i - c_j)| <= max_offset (plane-offset test). <= 0 disables.
 *   min_triangles  [tri_min] if > 0, segments of at most min_triangles triangles are dropped
 *                  (Algorithm 5 keeps |T^g_i| > tri_min).
 *   flags          0, or PL3D_FLAG_SEED_PTP: region growing as Algorithm 5 orders it, with
 *                  max_offset (> 0 required) as ptp_max read seed-relative. Seeds are taken in
 *                  GID order; a segment is its seed plus every triangle reachable through twin
 *                  half-edges over triangles of the seed's group that are in no segment yet and
 *                  whose centroid lies within ptp_max of the plane through the seed's centroid
 *                  with the group's dominant normal; a dropped segment's triangles stay consumed;
 *                  labels are still each segment's smallest GID (its seed). The GPU labels the
 *                  order-independent components and flags those leaving their seed's slab; the
 *                  host regrows only the flagged ones, so such calls synchronise the stream.
 *                  Single-frame entry points only (batches, the server and the allocation-free
 *                  entry return PL3D_ERR_UNSUPPORTED).
 */
#define PL3D_FLAG_SEED_PTP 1u
typedef struct pl3d_params {
    int32_t lap_iters;
    float lap_lambda;
    int32_t lap_kernel;
    int32_t bil_iters;
    float bil_sigma_len;
    float bil_sigma_ang;
    int32_t bil_kernel;
    float max_edge;
    float min_dot;
    float max_offset;
    int32_t min_triangles;
    uint32_t flags;
} pl3d_params;

/* Fills *p with the RGBD settings of the paper's RealSense experiment (Section 9.3.1):
 * 2 Laplacian iterations (lambda 1, kernel 3), 2 bilateral iterations (sigma_c 0.1,
 * sigma_s 0.15, kernel 3), l_max 0.05, ang_min 0.96; max_offset and tri_min off.
 * Returns PL3D_ERR_INVALID_ARG if p is NULL. Host only. */
int pl3d_default_params(pl3d_params* p);

/* Host-only argument check shared by every entry point: H, W >= 2, 2(H-1)(W-1) < 2^31,
 * K in [1, 254], finite and non-zero dominant normals (host pointer, may be NULL to skip
 * that check), parameter ranges as documented above. No CUDA call. */
int pl3d_validate(const pl3d_params* params, int H, int W, const float* dominant_normals, int K);

/* Creates a context bound to CUDA device `cuda_device` (the device must be sm_103-class,
 * else PL3D_ERR_UNSUPPORTED). The context owns scratch memory that grows to the largest
 * frame seen (growth synchronises the stream of the call that grows it): displacements,
 * groups, the grid-barrier and error words, and the counters with which the tiles of one
 * launch decide which of two neighbours joins their shared border. Calls on one context run
 * one after another: enqueue them on one stream (or order their streams), and use a context
 * per concurrent stream or thread. *out receives the context; on error *out is NULL. */
int pl3d_create(pl3d_ctx** out, int cuda_device);

/* Releases the context and its scratch memory after synchronising its device.
 * NULL is ignored. */
void pl3d_destroy(pl3d_ctx* ctx);

/*
 * Runs the whole path on one frame, asynchronously on `stream` (a cudaStream_t; NULL =
 * the legacy default stream).
 *   points            device, H*W*3 FP32, row-major xyz, not modified.
 *   dominant_normals  host, K*3 FP32; normalised by the library; read before return.
 *   out_tri_mask      device, 2(H-1)(W-1) bytes: 1 = triangle kept (all vertices valid and
 *                     longest edge <= max_edge), else 0.
 *   out_normals       device, 2(H-1)(W-1)*3 FP32: filtered unit normal; NaN where the
 *                     triangle has an invalid vertex or a degenerate (zero-area) shape.
 *   out_labels        device, 2(H-1)(W-1) int32: the smallest GID of the triangle's planar
 *                     segment, or -1 (no group, or a segment of at most min_triangles).
 * The caller owns every buffer; the library keeps no pointer after the call returns and
 * reads/writes them only in work enqueued on `stream`. Outputs are complete when the
 * stream reaches this call's end. Buffers must not overlap.
 */
int pl3d_extract_planes(pl3d_ctx* ctx, const float* points, int H, int W, const pl3d_params* params,
                        const float* dominant_normals, int K, uint8_t* out_tri_mask, float* out_normals,
                        int32_t* out_labels, void* stream);

/* As pl3d_extract_planes, plus two optional device outputs (NULL = not written):
 *   out_points  H*W*3 FP32 smoothed points (invalid points NaN);
 *   out_groups  2(H-1)(W-1) bytes, the group of Algorithm 4 (255 = none). */
int pl3d_extract_planes_ex(pl3d_ctx* ctx, const float* points, int H, int W, const pl3d_params* params,
                           const float* dominant_normals, int K, uint8_t* out_tri_mask, float* out_normals,
                           int32_t* out_labels, float* out_points, uint8_t* out_groups, void* stream);

/* As pl3d_extract_planes with HOST buffers: copies points to the device, runs the path on
 * `stream` and brings the three outputs back, then synchronises the stream before
 * returning. Page-locked host buffers make the copies asynchronous DMA; pageable ones work
 * but are slower. A page-locked mask or labels buffer that the device can address is written
 * by the kernel itself (the mask as each tile finishes, the final labels by the last label
 * phase). The path runs as two launches here: once mask, normals and groups are final, the
 * normals are copied out on a stream of the context while the second launch joins the
 * segments across tiles. The results are the same either way. Device staging buffers and the
 * copy stream are owned by the context. */
int pl3d_extract_planes_host(pl3d_ctx* ctx, const float* host_points, int H, int W, const pl3d_params* params,
                             const float* dominant_normals, int K, uint8_t* host_tri_mask, float* host_normals,
                             int32_t* host_labels, void* stream);

/*
 * Pipelined host-buffer frames (no counterpart in the paper): a stream of frames from host
 * memory, each through the same path as pl3d_extract_planes, with the copies of one frame
 * overlapping the kernels of the others. A pipeline owns a context, three CUDA streams (input
 * copies, kernels, output copies) and `depth` sets of device buffers for frames of up to
 * max_points points. The kernels run one frame at a time in submission order on the kernel
 * stream (they share the context's scratch); a frame's input copy runs while the frames before
 * it are in their kernels, and its output copy while the frames after it are.
 *
 * pl3d_pipeline_create   device: CUDA device; max_points: largest H * W submitted (>= 4);
 *                        depth: frames in flight, 1 .. 16. Allocates everything up front
 *                        (PL3D_ERR_OUT_OF_MEMORY when that fails); *out NULL on failure.
 * pl3d_pipeline_submit   enqueues one frame and returns its ticket (1, 2, 3, ...) without
 *                        waiting for it. Arguments as pl3d_extract_planes_host; the host
 *                        buffers should be page-locked (pageable ones make the copies
 *                        synchronous), must stay valid and untouched until the frame is waited
 *                        for, and must not overlap. When `depth` frames are in flight it first
 *                        waits for the oldest (its status is kept for pl3d_pipeline_wait).
 *                        PL3D_FLAG_SEED_PTP is not supported (PL3D_ERR_UNSUPPORTED); H * W
 *                        above max_points is PL3D_ERR_INVALID_ARG. A failed submit issues no
 *                        ticket (an input copy it enqueued lands in a free buffer set).
 * pl3d_pipeline_wait     waits until the frame's three outputs are in host memory and returns
 *                        its status: PL3D_OK, or PL3D_ERR_TIMEOUT when a bounded device wait gave
 *                        up during it or during a frame whose kernels overlapped its output copy
 *                        (their results are void; the context's error word and grid-barrier
 *                        state are cleared after every stream has drained). Frames complete in
 *                        submission order. A ticket waited for before returns its kept status
 *                        while it is among the last 1024 issued; an unknown or older ticket is
 *                        PL3D_ERR_INVALID_ARG.
 * pl3d_pipeline_destroy  waits for every frame in flight and frees everything (NULL is a no-op).
 */
typedef struct pl3d_pipeline pl3d_pipeline;
int pl3d_pipeline_create(int device, int64_t max_points, int depth, pl3d_pipeline** out);
int pl3d_pipeline_submit(pl3d_pipeline* pl, const float* host_points, int H, int W, const pl3d_params* params,
                         const float* dominant_normals, int K, uint8_t* host_tri_mask, float* host_normals,
                         int32_t* host_labels, uint64_t* ticket);
int pl3d_pipeline_wait(pl3d_pipeline* pl, uint64_t ticket);
int pl3d_pipeline_destroy(pl3d_pipeline* pl);
/* The pipeline's context, owned by the pipeline (NULL for NULL): for pl3d_set_timing,
 * pl3d_read_timing, pl3d_launch_count and pl3d_selftest_wait_timeout while no frame is in flight.
 * An error word set between frames is reported by the next frame submitted. */
pl3d_ctx* pl3d_pipeline_context(pl3d_pipeline* pl);

/* Waits for `stream` and reports any pending CUDA error as PL3D_ERR_CUDA. Then reads the
 * context's device error word: when a bounded device wait of an earlier call gave up (a grid
 * barrier or a TMA copy not completing within 1 s), the results of the calls since the last
 * pl3d_sync are void; the word and the grid-barrier state are cleared and PL3D_ERR_TIMEOUT is
 * returned, after which the context runs new calls normally. */
int pl3d_sync(pl3d_ctx* ctx, void* stream);

/* Self-test of the device-side timeout path (no counterpart in the paper). Enqueues on `stream`
 * one small cooperative kernel that makes one of the library's bounded waits run out, with the
 * limit limit_ns (1e5 .. 1e10 nanoseconds) instead of 1 s:
 *   kind 1  the grid barrier of the path's kernels, in a grid of two CTAs one of which returns
 *           without arriving;
 *   kind 2  an mbarrier of the kind TMA copies complete on, which nothing arms (no copy issued).
 * The waiting thread records the timeout in the device error word of `ctx` -- or, with ctx NULL,
 * in that of the allocation-free entry point on the current device -- and returns; nothing
 * faults, traps or waits without bound. The next pl3d_sync(ctx, stream) (pl3d_static_sync(stream)
 * for NULL) then returns PL3D_ERR_TIMEOUT and clears the words. Returns PL3D_ERR_INVALID_ARG for
 * another kind or limit, else the launch status. */
int pl3d_selftest_wait_timeout(pl3d_ctx* ctx, int kind, int64_t limit_ns, void* stream);

/* Static, human-readable text for a status code. Never NULL. */
const char* pl3d_status_string(int status);

/* Per-kernel timing (CUDA events recorded around each launch, on the launch stream).
 * pl3d_set_timing(ctx, 1) starts recording; pl3d_read_timing waits for the recorded events,
 * writes per-phase total milliseconds and launch counts for up to n_slots phases
 * (ms_out, launches_out may be NULL) and returns the number of phases (PL3D_TIMING_SLOTS),
 * clearing the totals when reset != 0. Phase order: see pl3d_timing_slot_name. Slots 0-3 are
 * wall times of the phases (the device clock read by one CTA at each phase boundary; the
 * single-iteration Laplacian kernel's own span counts as the Laplacian phase); slots 4-7 are CUDA
 * event times of whole launches and copies; slots 8-12 ("..._cta") are the bilateral tiles' time
 * in each stage -- staging, geometry, iterations, finish, tile labels -- summed over tiles (CTA
 * time, not wall time: their shares split the bilateral phase). */
#define PL3D_TIMING_SLOTS 13
int pl3d_set_timing(pl3d_ctx* ctx, int enable);
int pl3d_read_timing(pl3d_ctx* ctx, double* ms_out, int64_t* launches_out, int n_slots, int reset);
const char* pl3d_timing_slot_name(int slot);

/* Number of kernels this context has launched since it was created. */
int64_t pl3d_launch_count(const pl3d_ctx* ctx);

/*
 * Allocation-free entry point. The paper has no counterpart: this serves callers that cannot
 * allocate device memory while they run -- a real-time sensor loop that must avoid the
 * device-wide synchronisation cudaMalloc/cudaFree can cause, a process whose memory budget
 * was fixed at start-up, or a plugin that receives a stream and buffers per call and keeps
 * no context. Same arguments, results and errors as pl3d_extract_planes, without a context:
 * the scratch comes from one fixed device array inside the library, which every GPU that
 * loads the library's kernels holds (pl3d_static_scratch_bytes(), about 10.4 MB) until the
 * process exits.
 *   - Frames are limited to H*W <= PL3D_STATIC_MAX_POINTS points (640 x 480) and to
 *     bil_iters <= 6 / (bil_kernel / 2); larger requests return PL3D_ERR_INVALID_ARG before
 *     anything is enqueued.
 *   - It never calls cudaMalloc, cudaFree or any allocating routine.
 *   - The first call on a device (the current device) looks up the array's device address
 *     and configures the kernels; make that first call before any stream capture.
 *   - Every call uses the same array: calls whose work overlaps on the GPU race and must be
 *     serialised by the caller. Nothing needs clearing between calls that succeed.
 *   - Device-side errors (a bounded wait that gave up) are recorded in the array's error word;
 *     pl3d_static_sync reports them. Call it after the calls whose results you use.
 */
#define PL3D_STATIC_MAX_POINTS 307200
int pl3d_extract_planes_static(const float* points, int H, int W, const pl3d_params* params,
                               const float* dominant_normals, int K, uint8_t* out_tri_mask, float* out_normals,
                               int32_t* out_labels, void* stream);
/* Bytes of device memory the allocation-free entry point reserves on every GPU. */
size_t pl3d_static_scratch_bytes(void);
/* pl3d_sync for the allocation-free entry point on the current device: waits for `stream`,
 * reports a pending CUDA error as PL3D_ERR_CUDA, then reads the array's device error word. When
 * a bounded wait of a call since the last check gave up, those calls' results are void: the
 * error word and the grid-barrier words are cleared (a memset into the same array, enqueued on
 * `stream` and waited for) and PL3D_ERR_TIMEOUT is returned; later calls run normally. Allocates
 * nothing. */
int pl3d_static_sync(void* stream);

/*
 * Batches. The paper runs its pipeline one frame at a time; a batch runs the whole path of
 * pl3d_extract_planes_ex (same arguments per frame, same results bit for bit) on many frames
 * of any sizes in ONE persistent cooperative launch, replayed from a CUDA graph. Each phase
 * (Laplacian tiles, bilateral tiles, tile-border merge, labels) spans the work of all frames,
 * so small frames no longer leave most of the GPU idle.
 *
 * pl3d_frame describes one frame; pointers and sizes as in pl3d_extract_planes_ex (points and
 * outputs on the device, params and dominant_normals on the host; out_points and out_groups
 * may be NULL). Frames of one batch may differ in size, iteration counts and thresholds, but
 * every frame with lap_iters > 0 must use one lap_kernel and every frame with bil_iters > 0 one
 * bil_kernel (else PL3D_ERR_UNSUPPORTED). Output buffers of different frames must not overlap.
 *
 * pl3d_extract_planes_batched enqueues the batch on `stream`. Host work: it validates every
 * frame (any invalid frame rejects the whole batch before anything is enqueued), fills a
 * descriptor block in page-locked memory and copies it to the device unless it is identical to
 * the last one, then launches the graph for the batch's launch shape (built on first use).
 * Scratch for all frames of the batch comes from one slab of the context that grows to the
 * largest batch (growth synchronises the stream). n == 0 does nothing. Calls are ordered on
 * the stream like every other call on the context.
 */
typedef struct pl3d_frame {
    const float* points;
    int32_t H;
    int32_t W;
    const pl3d_params* params;
    const float* dominant_normals;
    int32_t K;
    uint8_t* out_tri_mask;
    float* out_normals;
    int32_t* out_labels;
    float* out_points;
    uint8_t* out_groups;
} pl3d_frame;

int pl3d_extract_planes_batched(pl3d_ctx* ctx, const pl3d_frame* frames, int n, void* stream);

/*
 * Launch shape of every later call on the context (single frames and batches). None of these
 * changes a result bit: iterations split over more passes go through global memory as the same
 * FP32 values the fused form keeps in shared memory.
 *   lap_fuse     most Laplacian iterations fused into one tile pass (0 = as many as the tile's
 *                halo of 8 points allows); fewer means smaller halos but more passes.
 *   bil_fuse     the same for the bilateral (halo of 6 quads).
 *                Either depth is raised where needed so that a filter takes at most 8 passes.
 *   ctas_per_sm  resident CTAs per SM of the persistent launch (0 = as many as fit, at most 2).
 *   lap_tile_h   Laplacian tile height in points, a multiple of 8 in [16, 64] (0 = 32, or 64 for a
 *                single-iteration first pass); tiles are 32 points wide. A height whose buffers
 *                would not fit two CTAs per SM for a pass falls back to 32 for that pass.
 *   bil_tile_h   bilateral tile height in quads, a multiple of 8 in [8, 32] (0 = 32); tiles are
 *                32 quads wide (a warp labels one tile row).
 * Smaller tiles spread a frame over more CTAs (more tiles per CTA to balance their costs) at the
 * price of more halo per output. pl3d_set_tuning(ctx, NULL) restores the defaults (all 0).
 * Negative fields and other tile heights are rejected with PL3D_ERR_INVALID_ARG.
 */
typedef struct pl3d_tuning {
    int32_t lap_fuse;
    int32_t bil_fuse;
    int32_t ctas_per_sm;
    int32_t lap_tile_h;
    int32_t bil_tile_h;
} pl3d_tuning;

int pl3d_set_tuning(pl3d_ctx* ctx, const pl3d_tuning* tuning);
int pl3d_get_tuning(const pl3d_ctx* ctx, pl3d_tuning* tuning);

/*
 * Autotuner: times the batch under launch shapes, `reps` timed runs each after one untimed run,
 * on `stream` with CUDA events, and keeps the fastest median as the context's tuning. It searches
 * in two stages: first the fused depths (1, 2 or 3 passes per filter, and one iteration per
 * Laplacian pass when its window is 3 x 3) x 1 or 2 CTAs per SM at the default tile shapes, then,
 * at the best of those, the tile heights (Laplacian 16, 32, 48, 64 points; bilateral 16, 24, 32
 * quads; 32 wide). Writes the choice to *best and its median milliseconds to *best_ms (either may be
 * NULL). Runs the batch (1 + reps) times per candidate and once more under the choice, so the
 * outputs hold that run's (identical) results. Synchronises the stream. reps in [1, 50].
 */
int pl3d_autotune_batched(pl3d_ctx* ctx, const pl3d_frame* frames, int n, void* stream, int reps,
                          pl3d_tuning* best, double* best_ms);

/* Counters of the batch machinery: graph launches, descriptor uploads (a batch identical to
 * the previous one skips its upload) and graphs instantiated. Any pointer may be NULL. */
int pl3d_batch_stats(const pl3d_ctx* ctx, int64_t* graph_launches, int64_t* desc_uploads, int64_t* graphs);

/*
 * Serving (no counterpart in the paper). A server takes frames from any number of sensors as
 * they arrive and runs them with continuous batching: a worker thread owns `max_inflight`
 * slots, each with its own stream, context and device arena; whenever a slot is free it takes
 * the waiting requests in arrival order, as many as its arena has room for (admission by free
 * HBM) up to `max_batch_frames`, copies their points in, runs them as one batch
 * (pl3d_extract_planes_batched) and copies the outputs back, while the other slot's batch is
 * still on the GPU. Two batches in flight run side by side, one CTA per SM each.
 *
 *   device            CUDA device (sm_103-class).
 *   max_inflight      1 or 2 batches on the GPU at once.
 *   max_batch_frames  1..4096 frames per launch; 1 = one plain single-frame launch per request
 *                     (with max_inflight 1: the plain sequential path).
 *   hbm_bytes         device memory for request buffers and scratch over all slots; 0 = half of
 *                     the free memory at creation. A slot holds hbm_bytes / max_inflight.
 *
 * pl3d_server_submit enqueues one frame and returns at once with a ticket (1, 2, 3, ... in
 * submission order). Host buffers as in pl3d_extract_planes_host (page-locked ones give
 * asynchronous copies); they stay the caller's and must stay valid and untouched until the
 * ticket completes. params and dominant_normals are copied. A frame that does not fit an empty
 * slot is rejected with PL3D_ERR_OUT_OF_MEMORY; invalid arguments with their error; nothing is
 * enqueued then. Results are bit-identical to pl3d_extract_planes on the same frame.
 *
 * pl3d_server_poll moves up to `max` completions to `out` (oldest first), waiting up to
 * wait_ms milliseconds for the first one (0 = do not wait, < 0 = until one arrives or nothing
 * is outstanding), and returns how many it wrote, or a negative error. A completion gives the
 * ticket, the status of its batch, the frames of that batch, the latency from submission to
 * the end of the batch's last copy (measured on the host when the stream reaches it) and the
 * time the request waited before its batch was enqueued.
 * pl3d_server_drain waits until every submitted request has completed.
 * pl3d_server_destroy drains, stops the worker and frees everything.
 */
typedef struct pl3d_server pl3d_server;

typedef struct pl3d_server_config {
    int32_t device;
    int32_t max_inflight;
    int32_t max_batch_frames;
    int32_t reserved;     /* must be 0 */
    int64_t hbm_bytes;
} pl3d_server_config;

typedef struct pl3d_completion {
    uint64_t ticket;
    int32_t status;
    int32_t batch_frames;
    double latency_ms;
    double queue_ms;
} pl3d_completion;

typedef struct pl3d_server_stats {
    int64_t submitted;
    int64_t completed;
    int64_t rejected;
    int64_t batches;
    int64_t triangles;            /* of completed requests */
    int64_t max_batch_frames;     /* largest batch launched */
    int64_t max_inflight;         /* most batches seen in flight at once */
    int64_t slot_bytes;           /* device bytes per slot (arena + scratch) */
} pl3d_server_stats;

int pl3d_server_create(pl3d_server** out, const pl3d_server_config* cfg);
int pl3d_server_submit(pl3d_server* srv, const float* host_points, int H, int W, const pl3d_params* params,
                       const float* dominant_normals, int K, uint8_t* host_tri_mask, float* host_normals,
                       int32_t* host_labels, uint64_t* ticket);
int pl3d_server_poll(pl3d_server* srv, pl3d_completion* out, int max, int wait_ms);
int pl3d_server_drain(pl3d_server* srv);
int pl3d_server_get_stats(const pl3d_server* srv, pl3d_server_stats* out);
void pl3d_server_destroy(pl3d_server* srv);

/*
 * Trace replay on a server (no counterpart in the paper): submits requests at scheduled arrival
 * times from the calling thread, the way sensors would, collects their completions and reports
 * latency from each scheduled arrival to the end of its result's copy-out, so that a host-side
 * replay loop in another language does not add its own lag to the measured tail.
 *
 * A source is one sensor: n_variants page-locked host frames of H x W points (submitted in turn),
 * its parameters and dominant normals, and `ring` sets of host output buffers (page-locked), used
 * in turn; a request that would reuse a set still in flight waits for it first (counted as
 * submit lag). Request i arrives arrival_s[i] seconds after the replay starts (non-decreasing)
 * from source source_of[i]. Every source frame is submitted once and drained before the clock
 * starts (warm-up). The call returns after the last completion.
 *
 * The report: requests, completed, failed (completions with an error status), batches launched
 * and the largest batch and number of batches in flight during the replay; wall seconds from the
 * first scheduled arrival to the last completion; latency percentiles p50 / p90 / p99 / max and
 * the mean in milliseconds; Mtri/s over the wall time; achieved frames/s; mean frames per batch
 * over the requests; and the p99 of the submit lag (submission time minus scheduled arrival).
 * Returns PL3D_ERR_INVALID_ARG for bad arguments, else the first submit error, else PL3D_OK.
 */
typedef struct pl3d_replay_source {
    const float* const* host_points;   /* [n_variants] frames, H * W * 3 floats each */
    int32_t n_variants;
    int32_t H, W;
    int32_t K;
    const pl3d_params* params;
    const float* dominant_normals;      /* K * 3 */
    int32_t ring;                       /* output buffer sets */
    int32_t reserved;                   /* must be 0 */
    uint8_t* const* host_mask;          /* [ring] */
    float* const* host_normals;         /* [ring] */
    int32_t* const* host_labels;        /* [ring] */
} pl3d_replay_source;

typedef struct pl3d_replay_report {
    int64_t requests;
    int64_t completed;
    int64_t failed;
    int64_t batches;
    int64_t max_batch_frames;
    int64_t max_inflight;
    double seconds;
    double p50_ms, p90_ms, p99_ms, max_ms, mean_ms;
    double mtri_s;
    double achieved_fps;
    double mean_batch_frames;
    double submit_lag_p99_ms;
} pl3d_replay_report;

int pl3d_server_replay(pl3d_server* srv, const pl3d_replay_source* sources, int n_sources, const double* arrival_s,
                       const int32_t* source_of, int64_t n, pl3d_replay_report* report);

/*
 * Explicit half-edge mesh and segment lists of one frame, the inputs of polygon extraction
 * (Section 7.2), in one launch on `stream`:
 *   Algorithm 1: T, the triangles of T_FC whose three points are valid, in GID order, each as
 *                its three point indices (first = {p3, p2, p1}, second = {p1, p4, p3}), and
 *                T_map, the index into T of every GID (-1 for a triangle with an invalid point);
 *   Algorithm 2: HE, the twin of every half-edge 3 t + e of T (e-th edge of triangle t in the
 *                order above), -1 on a border;
 *   segments:    for the labels of pl3d_extract_planes (each label is the smallest GID of its
 *                segment), the segments in ascending label order (seg_labels), CSR offsets
 *                into seg_tris, and seg_tris, the T indices of each segment's triangles in
 *                ascending order;
 *   boundary:    border[t], bit e set when triangle t is in a segment and its half-edge 3 t + e
 *                has no twin or a twin in another segment (or in none): the boundary half-edges
 *                polygon extraction follows.
 * All buffers are on the device and owned by the caller (Q = (H-1)(W-1)):
 *   points [H W 3] FP32 (the frame's input: validity as everywhere in this library);
 *   labels [2Q] int32, or NULL (then only T, T_map, HE and counts[0] are produced, and the
 *          segment buffers may be NULL);
 *   out_T [3 * 2Q], out_Tmap [2Q], out_HE [3 * 2Q] int32; out_counts int64 [3] = {|T|,
 *   segments, triangles in segments}; out_seg_labels [2Q], out_seg_offsets [2Q + 1],
 *   out_seg_tris [2Q] int32; out_border [2Q] uint8 or NULL.
 * Only the first counts[...] entries of each output are written. Sizes need 6 Q < 2^31 (half-edge
 * ids are int32), else PL3D_ERR_INVALID_ARG. The context's mesh scratch (about 28 bytes per
 * triangle) grows to the largest frame seen. Results are exact: no floating-point arithmetic.
 */
int pl3d_extract_mesh(pl3d_ctx* ctx, const float* points, const int32_t* labels, int H, int W, int32_t* out_T,
                      int32_t* out_Tmap, int32_t* out_HE, int64_t* out_counts, int32_t* out_seg_labels,
                      int32_t* out_seg_offsets, int32_t* out_seg_tris, uint8_t* out_border, void* stream);

/*
 * Fast Gaussian Accumulator (Section 6): dominant plane normals from the triangle normals,
 * replacing given dominant normals.
 *
 * Cells (Section 6.1.1): the faces of an icosahedron refined `level` times (0..5: 20 4^level
 * cells). Level 0 has the 12 unit vertices (-1, phi, 0), (1, phi, 0), (-1, -phi, 0),
 * (1, -phi, 0), (0, -1, phi), (0, 1, phi), (0, -1, -phi), (0, 1, -phi), (phi, 0, -1),
 * (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1) (before scaling, in this order) and the 20 faces made
 * by the triples of mutually adjacent vertices, in lexicographic order of the sorted triple,
 * counter-clockwise from outside. Level l + 1 splits face p = (a, b, c) into faces 4p .. 4p + 3 =
 * (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca), midpoints projected onto the sphere. A
 * cell's surface normal is its flat face's unit normal.
 *
 * pl3d_fastga_cells (host only) writes the level's surface normals (host, cells * 3 floats) and
 * 1-ring neighbours (host, cells * 12 int32, ascending, -1 padded; either pointer may be NULL)
 * and returns the number of cells. It builds the level's tables, the device search's included,
 * and returns PL3D_ERR_UNSUPPORTED if they fail their construction check (every rotated cell
 * normal of face 0's neighbourhood on a cell normal, child numbers kept).
 *
 * pl3d_fastga integrates every stride-th triangle of `normals` (device, n * 3 FP32, e.g. the
 * out_normals of pl3d_extract_planes; Section 6.3's sampling) whose normal is finite and, when
 * `mask` (device, n bytes) is given, whose mask byte is non-zero: each goes to the cell whose
 * surface normal is closest (Section 6.1.3, Algorithm 3). out_counts (device, cells int32) receives
 * the histogram; out_cells (device, n int32, or NULL) the cell of every triangle, -1 where not
 * integrated (up to near ties of FP32 dot products: a cell whose surface normal is within 1e-6 of
 * the closest one's dot product may be chosen instead). The first call for a level in a process
 * builds the level's tables on the host (about 0.1 s at level 4, 1 s at level 5) and the first
 * call on a context uploads them (synchronously). One cooperative launch; it uses the context's
 * grid barrier, so a device wait that gives up is reported by pl3d_sync as for the path itself.
 * Returns PL3D_ERR_UNSUPPORTED if the level's tables fail their own construction check (not
 * expected for levels 0 .. 5).
 *
 * pl3d_fastga_peaks (host only) detects peaks in a histogram (host, cells int32): a cell whose
 * count is above v_min and not below any 1-ring neighbour's (a plateau keeps its lowest index),
 * the cell graph standing in for the paper's unwrapped image and its 3 x 3 peak test
 * (Section 6.2). Peaks whose surface normals are closer than d_peak are merged by single-linkage
 * agglomerative clustering into their count-weighted mean normal. Up to max_peaks clusters are
 * written by decreasing total count (out_normals host [max_peaks * 3], out_weights host or
 * NULL); returns how many were written.
 */
int pl3d_fastga_cells(int level, float* out_normals, int32_t* out_neighbors);
int pl3d_fastga(pl3d_ctx* ctx, const float* normals, const uint8_t* mask, int64_t n, int level, int stride,
                int32_t* out_counts, int32_t* out_cells, void* stream);
int pl3d_fastga_peaks(int level, const int32_t* counts, float v_min, float d_peak, int max_peaks, float* out_normals,
                      int64_t* out_weights);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int pl3d_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PL3D_H */

// pl3d_internal.cuh -- declarations shared by the frame kernel and the C ABI of libpl3d.
//
// Data layout in device memory (one frame of H x W points, Q = (H-1)(W-1) quads):
//   input points     AoS  float [H][W][3]     (caller's buffer)
//   displacements    AoS  float [H][W][3]     (scratch, ping-pong pair): a smoothed point is the
//                                              input point plus its displacement, kept as that
//                                              pair of floats (see df32.cuh)
//   bilateral carry  AoS  float [2Q][3]       (scratch, only when the bilateral iterations need
//                                              more than one tile pass)
//   groups           u8   [2Q]                (scratch or the caller's buffer)
//   labels           i32  [2Q]                (caller's buffer; doubles as the union-find parents)
//   segment sizes    i32  [2Q]                (scratch, only when tri_min > 0)
//   barrier, error   u32 [2], i32             (scratch: grid barrier state, device error word)
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pl3d.h"

namespace pl3d {

constexpr int kThreads = 256;    // threads per CTA
constexpr int kTile = 32;        // tile edge: 32 x 32 points (Laplacian) or quads (bilateral)
constexpr int kLapMaxHalo = 8;   // largest halo (fused iterations x radius) of one Laplacian pass
constexpr int kBilMaxHalo = 6;   // same for the bilateral
constexpr int kExactCap = 256;   // deferred exact-normal quads a bilateral tile lists (then inline)
// Shared memory per CTA that still lets two CTAs share an SM (the bilateral pass at halo 3 needs
// this much); a Laplacian pass stages as many boxes ahead as fit within it.
constexpr int kTwoCtaSmem = 114048;
constexpr int kLapMaxStages = 3;   // box buffers of a Laplacian pass: this tile's and up to 2 ahead
constexpr int kLapThinTileH = 64;  // tile height of a single-iteration first Laplacian pass
// Tile heights a tuning may ask for (tiles stay kTile wide): Laplacian 16..64 and bilateral
// 8..32 rows, multiples of 8.
constexpr int kLapMinTileH = 16, kLapMaxTileH = 64;
constexpr int kBilMinTileH = 8, kBilMaxTileH = kTile;

// Centroid given to a triangle without a normal: its bilateral weight underflows to
// exactly 0 against any real triangle, so it drops out of every sum without a branch.
constexpr float kAbsentCentroid = 1.0e30f;

// Squared cross-product length at or below which a triangle has no normal (|n| <= 1e-20).
constexpr float kDegenerateLen2 = 1.0e-40f;

// Coordinates of magnitude 1e18 or more are outside the supported range (their squared
// distances overflow FP32); such points are treated like non-finite ones: invalid.
constexpr float kMaxCoord = 1.0e18f;
__host__ __device__ __forceinline__ bool point_valid(float x, float y, float z) {
    return fabsf(x) < kMaxCoord && fabsf(y) < kMaxCoord && fabsf(z) < kMaxCoord;   // false for NaN and inf
}

// Finite stand-in for an invalid point inside the Laplacian's shared-memory tile.
constexpr float kInvalidCoord = 1.0e30f;

__host__ __device__ inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// Shared-memory buffers start on 128-byte boundaries (TMA destinations).
__host__ __device__ inline int align_floats(int n) { return (n + 31) & ~31; }

// Dominant normals, unit length, passed to kernels by value (3 KB, fits the parameter space).
struct Dominant {
    int K;
    float v[PL3D_MAX_GROUPS * 3];
};

// A staged box: rows x cols floats of an AoS array seen as H rows of 3W floats. cols is a
// multiple of 4 (16 bytes) and covers the tile's points plus up to 3 floats of alignment slack.
struct BoxGeom {
    int rows;
    int cols;
};

struct LapPhase {
    int iters;                     // Jacobi iterations fused in this pass
    int halo;                      // iters * radius
    int use_tma;                   // points staged by TMA (tm_pts_lap), else plain loads
    int stages;                    // box buffers (1..kLapMaxStages): TMA loads of the next stages - 1
                                   // tiles overlap this tile
    int tile_h;                    // tile height in points: the tuning's, else 32, or kLapThinTileH for a
                                   // single-iteration first pass (tiles are 32 points wide)
    int tiles;                     // tiles of this pass
    int dbufs;                     // displacement buffers: 1 for a single-iteration first pass, else 2
    BoxGeom box;                   // rows = tile_h + 2 halo + 3 (spare rows), cols >= 3 (32 + 2 halo) + 3
    const float* d_in;             // displacement after the previous pass, or nullptr (zero)
    float* d_out;                  // displacement after this pass
    float* export_points;          // optional AoS export of v0 + d (last pass only)
};

struct BilPhase {
    int iters;
    int halo;
    int use_tma;                   // points and displacement staged by TMA (tm_pts_bil, tm_disp_bil)
    BoxGeom box;                   // rows = bil_th + 2 halo + 1, cols >= 3 (32 + 2 halo + 1) + 3
    int first, last;               // first pass builds the normals; last pass finishes the quads
    const float* carry_in;         // AoS [2Q][3] normals from the previous pass (not first)
    float* carry_out;              // AoS [2Q][3] normals for the next pass (not last)
};

constexpr int kMaxPasses = 8;

// Timing words after the phase totals (phase_ns[0..3]): lap1 stamps at phase_ns + 4 .. + 6, the
// bilateral tiles' stage totals at phase_ns + kStageSlot .. + kStageSlot + kBilStages - 1.
constexpr int kStageSlot = 7;
constexpr int kBilStages = 5;

struct FrameArgs {
    CUtensorMap tm_pts_lap;        // points, Laplacian box (first pass)
    CUtensorMap tm_pts_bil;        // points, bilateral box
    CUtensorMap tm_disp_bil;       // final displacement, bilateral box
    const float* points;
    const float* disp;             // final displacement, read by the bilateral and the merge
    int H, W;
    float lambda;
    int n_lap;
    LapPhase lap[kMaxPasses];
    int n_bil;
    int bil_th;                    // bilateral tile height in quads (tiles are kTile = 32 quads wide)
    BilPhase bil[kMaxPasses];
    uint8_t* out_mask;
    float* out_normals;
    uint8_t* groups;
    int32_t* labels;
    int32_t* labels_copy;          // optional second destination of the final labels (for example
                                   // page-locked host memory), written by the last label phase
    int32_t* sizes;                // zeroed in the bilateral pass when tri_min > 0, else nullptr
    float c_scale;                 // sqrt(log2(e) / (2 sigma_c^2)): centroid pre-scale
    float a_norm;                  // log2(e) / sigma_s^2
    float max_edge2;               // l_max^2, or +inf when disabled
    float min_dot;
    float max_offset;              // <= 0 when disabled
    float max_offset_scaled;       // max_offset * c_scale
    int min_triangles;
    unsigned* barrier;             // [2] grid barrier state
    int* error;                    // device error word (sync.cuh bits)
    unsigned* border;              // [2 x bilateral tiles], even between launches: counters of the tile
                                   // borders that the bilateral tiles join themselves; nullptr: the
                                   // merge phase joins them
    unsigned long long* phase_ns;  // [4] accumulated phase times (then the lap1 stamps and the bilateral
                                   // stage totals, see kStageSlot), or nullptr
    int part;                      // 0: the whole path; 1: smoothing and tile-local segments only
                                   // (mask, normals, groups final); 2: the segments across tiles only
    Dominant nd;
};

template <int RL, int RB>
__global__ void frame_kernel(const __grid_constant__ FrameArgs a);

// A batch of frames in one persistent launch. Everything the kernel reads lives in one device
// block laid out for `cap` frames: a header, per-pass prefix sums of the frames' tile counts,
// prefix sums of their merge items and triangles, and one FrameArgs per frame (whose tensor
// maps are then read from global memory).
struct BatchHeader {
    int n;                         // frames in this batch
    int n_lap, n_bil;              // most Laplacian / bilateral passes of any frame
    int any_filter;                // some frame has tri_min > 0
    int timing;                    // accumulate phase times into BatchArgs::phase_ns
    int lap_buf[kMaxPasses];       // per Laplacian pass: floats of the largest box over the frames
    int lap_stages[kMaxPasses];    // per Laplacian pass: box buffers (1..kLapMaxStages)
    int lap_dbufs[kMaxPasses];     // per Laplacian pass: displacement buffers (1 or 2)
    int pad[3];
};

struct BatchArgs {
    const BatchHeader* hdr;
    const int* lap_tiles;          // [kMaxPasses][cap + 1]: pass c, frames before f -> tiles
    const int* bil_tiles;          // [kMaxPasses][cap + 1]
    const long long* merge_items;  // [cap + 1]
    const long long* tris;         // [cap + 1]
    const FrameArgs* frames;       // [cap], 64-byte aligned
    int stride;                    // cap + 1
    unsigned* barrier;
    int* error;
    unsigned long long* phase_ns;
};

template <int RL, int RB>
__global__ void batch_kernel(const __grid_constant__ BatchArgs b);

// The single-iteration Laplacian pass with a 3 x 3 window as a kernel of its own (lap1.cu): used
// when every Laplacian pass of a frame (of every frame of a batch) runs at most one iteration,
// before the persistent kernel, which then starts at the bilateral. Work unit: a warp task of
// kLap1Cols columns x kLap1Rows rows of one frame (a pair of columns per lane). Taller tasks (48
// rows) and a height chosen per launch to even out the last round of tasks both measured slower
// than 24 rows on the 256-frame batch.
constexpr int kLap1Cols = 64;
constexpr int kLap1Rows = 24;
// Threads per CTA, and CTAs per SM the register budget is set for (without, with the previous
// pass's displacement).
constexpr int kLap1Threads = 128;
constexpr int kLap1Ctas = 5;
constexpr int kLap1CtasD = 4;
__host__ __device__ inline int lap1_tasks(int H, int W) { return div_up(H, kLap1Rows) * div_up(W, kLap1Cols); }

struct Lap1Frame {
    const float* points;
    const float* d_in;             // previous pass's displacement, or nullptr (first pass)
    float* d_out;
    float* export_points;          // optional AoS export of v0 + d (last pass only)
    int H, W;
    int iters;                     // 0 (the displacement stays zero) or 1
    float lambda;
};

struct Lap1Args {
    Lap1Frame one;                 // the frame, when hdr == nullptr
    const BatchHeader* hdr;        // batch: frame count and timing flag, or nullptr
    const FrameArgs* frames;       // batch: pass `pass` of every frame
    const int* task_pre;           // batch: [n + 1] prefix sums of the frames' warp tasks in this pass
    int pass;
    unsigned long long* stamp;     // [3]: latest ~start, latest end, CTAs done; or nullptr (no timing)
    unsigned long long* phase_ns;  // the Laplacian span is added to phase_ns[0]
    unsigned* sched;               // [2], zero at rest: tasks handed out after the first round, CTAs
                                   // done (the last CTA puts both back to zero)
};

template <bool WITH_D>
__global__ void lap1_kernel(const __grid_constant__ Lap1Args a);

// --------------------------------------------------------------------------- host side

// Device buffers one frame needs besides its inputs and outputs.
struct FrameScratch {
    float* disp[2];                // >= 3 H W floats each, 16-byte aligned
    float* carry[2];               // >= 6 Q floats each when the bilateral needs several passes
    uint8_t* groups;               // >= 2 Q
    int32_t* sizes;                // >= 2 Q
    unsigned* barrier;             // [2], zero before the first use
    int* error;                    // [1]
    unsigned long long* phase_ns;  // [4] or nullptr
    unsigned* lap1_sched;          // [2], zero at rest: the single-iteration Laplacian's task counter
    unsigned* border;              // cap_border counters, zeroed when allocated, or nullptr
    size_t cap_border;
    uint8_t* seed_flags;           // >= 2 Q, PL3D_FLAG_SEED_PTP only
    float* seed_centroids;         // >= 6 Q, PL3D_FLAG_SEED_PTP only
};

// Launch-shape choices that leave every result bit-identical (Jacobi iterations split over
// more passes go through global memory as the same FP32 values).
struct Tuning {
    int lap_fuse;                  // most Laplacian iterations per pass, 0 = as many as fit the halo
    int bil_fuse;                  // same for the bilateral
    int ctas_per_sm;               // 0 = as many as fit
    int lap_tile_h;                // Laplacian tile height in points, 0 = 32 (64 for a single-iteration
                                   // first pass); a height whose buffers would not fit two CTAs per SM
                                   // falls back to 32
    int bil_tile_h;                // bilateral tile height in quads, 0 = 32
};

// Tile-border counters a frame's bilateral tiles use under tuning t (FrameArgs::border).
size_t border_counters(int H, int W, const Tuning& t);

// Number of bilateral passes the parameters need (> 1 needs the carry buffers).
int bilateral_passes(const pl3d_params* p, const Tuning& t);

// The frame's final displacement buffer among sc.disp (smoothed point = input point + it).
const float* final_disp(const FrameScratch& sc, const pl3d_params* p, const Tuning& t);

// PL3D_FLAG_SEED_PTP: turns the component labels of a frame (computed without offset test and
// tri_min) into Algorithm 5's seeded segments; synchronises the stream (pl3d_seeded.cu).
int seeded_labels(const FrameScratch& sc, const float* disp, const float* points, int H, int W, const pl3d_params* p,
                  const float* nd_host, int K, const uint8_t* groups, int32_t* labels, cudaStream_t s);

// Floats of one (aligned) buffer of a Laplacian pass with the given halo and tile height, the
// shared memory of such a pass with `stages` box buffers and `dbufs` displacement buffers, and the
// most stages (1..kLapMaxStages) that keep two CTAs per SM for buffers of `box_floats`.
int lap_box_floats(int halo, int tile_h);
size_t lap_smem_for(int box_floats, int stages, int dbufs);
int lap_stages_for(int box_floats, int dbufs);

// Dynamic shared memory the persistent kernels need for this frame under tuning t.
size_t frame_smem_bytes(const pl3d_params* p, const Tuning& t);

// Everything a launch needs besides the frame's arguments.
struct FramePlan {
    const void* frame_fn;          // frame_kernel<RL, RB>
    const void* batch_fn;          // batch_kernel<RL, RB>
    int rl, rb;
    size_t smem;                   // dynamic shared memory
    int tiles_lap, tiles_bil;      // tiles per pass
    long long merge_items;         // tile-border twins
    long long tris;                // 2 (H-1)(W-1)
};

// Fills the arguments of one frame (no CUDA call besides tensor-map encoding).
int frame_build(FrameArgs& a, FramePlan& plan, const FrameScratch& sc, const float* points, int H, int W,
                const pl3d_params* p, const float* nd_host, int K, uint8_t* out_mask, float* out_normals,
                int32_t* out_labels, float* out_points, uint8_t* out_groups, const Tuning& t,
                int32_t* out_labels_copy = nullptr);

// batch_kernel<rl, rb>, or nullptr outside radii 1..3.
const void* batch_kernel_for_radii(int rl, int rb);

// Resident CTAs of a kernel over the whole device for a shared-memory size (cached).
int resident_ctas(const void* fn, size_t smem, int dev, int threads = kThreads);

// Sets the shared-memory opt-in of every frame kernel on the current device.
cudaError_t frame_configure();

// lap1_kernel<WITH_D> (lap1.cu) and its dynamic shared memory.
const void* lap1_kernel_for(bool with_d);
size_t lap1_smem_bytes(bool with_d);

// Whether every Laplacian pass of these frame arguments runs at most one iteration with a 3 x 3
// window, so that lap1_kernel takes them.
bool lap1_eligible(const FrameArgs& a, int rl);

// Grid of a lap1 launch over `tasks` warp tasks (all resident CTAs when tasks < 0).
int lap1_grid(int dev, bool with_d, long long tasks);

// Enqueues the whole path for one frame on `s`: one cooperative launch, after one lap1_kernel launch
// per Laplacian pass when every pass runs at most one iteration with a 3 x 3 window. Returns a
// PL3D status. The timing stamps of lap1 launches sit after the phase totals (phase_ns + 4).
// With `normals_ready`, the path runs as two launches and the event is recorded between them,
// once mask, normals and groups are final (the segments across tiles come after it).
// *launches (optional) receives the number of kernels enqueued.
int frame_launch(const FrameScratch& sc, const float* points, int H, int W, const pl3d_params* p, const float* nd_host,
                 int K, uint8_t* out_mask, float* out_normals, int32_t* out_labels, float* out_points,
                 uint8_t* out_groups, const Tuning& t, cudaStream_t s, int32_t* out_labels_copy = nullptr,
                 cudaEvent_t normals_ready = nullptr, int* launches = nullptr);

// Device address of the allocation-free entry point's control words (barrier [2], error word,
// pad) on the current device (pl3d_static.cu).
int static_control_words(unsigned** ctl);

// Grid size of a persistent launch: all resident CTAs (or ctas_per_sm per SM), at most `work`.
int persistent_grid(const void* fn, size_t smem, int dev, const Tuning& t, long long work);

}  // namespace pl3d

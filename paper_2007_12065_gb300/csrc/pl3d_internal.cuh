// pl3d_internal.cuh -- declarations shared by the kernels and the C ABI of libpl3d.
//
// Data layout in device memory (one frame of H x W points, Q = (H-1)(W-1) quads):
//   input points     AoS  float [H][W][3]            (caller's buffer)
//   displacements    SoA  float dx[H*W], dy[H*W], dz[H*W] (context scratch, ping-pong pair):
//                    a smoothed point is the input point plus its displacement, kept as
//                    that pair of floats (see df32.cuh)
//   bilateral carry  AoS  float [2Q][3]               (context scratch, only when the
//                                                      bilateral iterations need more than
//                                                      one launch)
//   groups           u8   [2Q]                        (context scratch or caller's buffer)
//   labels           i32  [2Q]                        (caller's buffer; doubles as the
//                                                      union-find parent array)
//   segment sizes    i32  [2Q]                        (context scratch, only when tri_min > 0)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pl3d.h"

namespace pl3d {

// Largest supported filter radius (kernel size 7).
constexpr int kMaxRadius = 3;

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

// Dominant normals, unit length, passed to kernels by value (3 KB, fits the parameter space).
struct Dominant {
    int K;
    float v[PL3D_MAX_GROUPS * 3];
};

// ---------------------------------------------------------------- Laplacian (Eq. 1-2)
struct LapArgs {
    const float* points;                      // AoS input points (the v0 of every launch)
    const float* in_dx;                       // displacement after the previous launch, or
    const float* in_dy;                       // nullptr for the first launch (zero)
    const float* in_dz;
    float* out_dx;                            // displacement after this launch, SoA
    float* out_dy;
    float* out_dz;
    float* out_aos;                           // optional AoS export of v0 + d (rounded)
    int H, W;
    int iters;                                // iterations fused in this launch (>= 0)
    float lambda;
};
// Tile of output points per CTA.
constexpr int kLapTileH = 32;
constexpr int kLapTileW = 32;
constexpr int kLapThreads = 256;
// Largest halo (fused iterations x radius) one launch may carry.
constexpr int kLapMaxHalo = 8;
cudaError_t launch_laplacian(const LapArgs& a, int radius, cudaStream_t s);
// Opts the kernels in to their largest shared-memory size on the current device.
cudaError_t laplacian_configure();
size_t laplacian_smem_bytes(int radius, int iters);

// ------------------- normals + bilateral (Eq. 3-6) + Algorithm 4 + tile-local Algorithm 5
struct BilArgs {
    const float* points;                      // AoS input points v0
    const float* dx;                          // displacements, SoA (smoothed = v0 + d)
    const float* dy;
    const float* dz;
    const float* carry_in;                    // AoS [2Q][3] normals from the previous launch (non-first)
    float* carry_out;                         // AoS [2Q][3] normals for the next launch (non-last)
    uint8_t* out_mask;                        // last launch only
    float* out_normals;
    uint8_t* out_groups;
    int32_t* out_labels;                      // GID of the tile-local root, or -1
    int32_t* sizes;                           // zeroed for the merge/flatten passes, or nullptr
    int H, W;
    int iters;                                // iterations fused in this launch (>= 0)
    float c_scale;                            // sqrt(log2(e) / (2 sigma_c^2)): centroid pre-scale
    float a_norm;                             // log2(e) / sigma_s^2
    float max_edge2;                          // l_max^2, or +inf when disabled
    float min_dot;
    float max_offset_scaled;                  // max_offset * c_scale, <= 0 when disabled
    Dominant nd;
};
constexpr int kBilTileH = 32;                 // quads per CTA tile
constexpr int kBilTileW = 32;
constexpr int kBilThreads = 256;
constexpr int kBilMaxHalo = 6;
cudaError_t launch_bilateral(const BilArgs& a, int radius, bool first, bool last, cudaStream_t s);
cudaError_t bilateral_configure();
size_t bilateral_smem_bytes(int radius, int iters);
// Host-side scale factors of the bilateral weights, kept finite and non-zero.
void bilateral_scales(float sigma_c, float sigma_s, int iters, float* c_scale, float* a_norm);

// ------------------------------------------- segments across tile borders (Algorithm 5)
struct LabelArgs {
    const uint8_t* groups;
    int32_t* labels;                          // tile-local roots in, labels out
    int32_t* sizes;                           // segment sizes (tri_min > 0) or nullptr
    const float* points;                      // AoS input points and SoA displacements
    const float* dx;                          // (offset test only)
    const float* dy;
    const float* dz;
    int H, W;
    int tile_h, tile_w;                       // the bilateral kernel's tile, in quads
    float max_offset;                         // <= 0: no offset test
    int min_triangles;
    Dominant nd;
};
cudaError_t launch_label_merge(const LabelArgs& a, cudaStream_t s);
cudaError_t launch_label_flatten(const LabelArgs& a, cudaStream_t s);
cudaError_t launch_label_filter(const LabelArgs& a, cudaStream_t s);

__host__ __device__ inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace pl3d

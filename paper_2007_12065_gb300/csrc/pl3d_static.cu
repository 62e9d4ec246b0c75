// pl3d_static.cu -- pl3d_extract_planes_static: the whole path without any allocation.
//
// Who needs it: code that must not allocate device memory after start-up -- a real-time
// sensor loop that has to avoid the device-wide synchronisation cudaMalloc/cudaFree can
// cause, a process whose memory budget was fixed when it started, or a caller with no
// context object to keep (plugins that get a stream and buffers per call). Such a caller
// passes its inputs and outputs; the scratch the path needs (point displacements, groups,
// segment sizes) lives in the file-scope device array below instead of in a context.
//
// The array is part of the library's device code, so every GPU on which the library's
// kernels load holds it (static_scratch_bytes(), about 10.4 MB) until the process exits.
// Host code cannot use the array's name as a device address: the first call on a device
// looks the address up with cudaGetSymbolAddress (with that device current), checks the
// device and sets the kernels' shared-memory limits; later calls reuse the result. Make
// that first call before any stream capture on the device.
//
// All calls share the one array: calls whose work overlaps on the GPU (different streams,
// or host threads that do not order their streams) race on it and must be serialised by
// the caller. Nothing in it needs clearing between calls -- every scratch value is written
// before it is read within a call.
#include <float.h>
#include <math.h>

#include <mutex>

#include "pl3d_internal.cuh"

using namespace pl3d;

namespace {

constexpr size_t kMaxPoints = PL3D_STATIC_MAX_POINTS;
constexpr size_t kMaxTri = 2 * kMaxPoints;                       // 2(H-1)(W-1) < 2 H W
constexpr size_t kDispBytes = 6 * kMaxPoints * sizeof(float);    // displacement ping-pong, SoA
constexpr size_t kGroupBytes = (kMaxTri + 255) / 256 * 256;
constexpr size_t kSizeBytes = kMaxTri * sizeof(int32_t);
constexpr size_t kScratchBytes = kDispBytes + kGroupBytes + kSizeBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool done = false;
    int status = PL3D_OK;
    unsigned char* scratch = nullptr;   // device address of g_static_scratch on this device
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current.
int setup_device(int dev, unsigned char** scratch) {
    if (dev < 0 || dev >= kMaxDevices) return PL3D_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_CUDA;   // not cached: a later call may succeed
        }
        if (prop.major != 10 || prop.minor != 3) {
            s.status = PL3D_ERR_UNSUPPORTED;
        } else if (cudaGetSymbolAddress((void**)&s.scratch, g_static_scratch) != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_CUDA;
        } else if (laplacian_configure() != cudaSuccess || bilateral_configure() != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_CUDA;
        } else {
            s.status = PL3D_OK;
        }
        s.done = true;
    }
    *scratch = s.scratch;
    return s.status;
}

}  // namespace

extern "C" size_t pl3d_static_scratch_bytes(void) { return kScratchBytes; }

extern "C" int pl3d_extract_planes_static(const float* points, int H, int W, const pl3d_params* p,
                                          const float* nd_host, int K, uint8_t* out_mask, float* out_normals,
                                          int32_t* out_labels, void* stream) {
    if (!points || !nd_host || !out_mask || !out_normals || !out_labels) return PL3D_ERR_INVALID_ARG;
    int rc = pl3d_validate(p, H, W, nd_host, K);
    if (rc != PL3D_OK) return rc;
    if ((size_t)H * (size_t)W > kMaxPoints) return PL3D_ERR_INVALID_ARG;
    const int br = p->bil_iters > 0 ? p->bil_kernel / 2 : 1;
    if (p->bil_iters > kBilMaxHalo / br) return PL3D_ERR_INVALID_ARG;   // would need the carry buffers
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    unsigned char* scratch = nullptr;
    if ((rc = setup_device(dev, &scratch)) != PL3D_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    float* disp = (float*)scratch;
    uint8_t* groups = scratch + kDispBytes;
    int32_t* sizes = (int32_t*)(scratch + kDispBytes + kGroupBytes);
    const size_t npts = (size_t)H * W;
    float* buf[2][3];
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k < 3; ++k) buf[b][k] = disp + (size_t)(3 * b + k) * npts;

    Dominant nd;
    nd.K = K;
    for (int j = 0; j < K; ++j) {
        const double x = nd_host[3 * j], y = nd_host[3 * j + 1], z = nd_host[3 * j + 2];
        const double len = sqrt(x * x + y * y + z * z);
        nd.v[3 * j] = (float)(x / len);
        nd.v[3 * j + 1] = (float)(y / len);
        nd.v[3 * j + 2] = (float)(z / len);
    }

    // Laplacian launches (displacement ping-pong in the static array).
    const int lr = p->lap_iters > 0 ? p->lap_kernel / 2 : 1;
    const int lfuse = kLapMaxHalo / lr;
    int remaining = p->lap_iters, cur = 0;
    bool first = true;
    do {
        const int it = remaining < lfuse ? remaining : lfuse;
        LapArgs la{};
        la.points = points;
        la.in_dx = first ? nullptr : buf[cur][0];
        la.in_dy = first ? nullptr : buf[cur][1];
        la.in_dz = first ? nullptr : buf[cur][2];
        const int nb = first ? cur : 1 - cur;
        la.out_dx = buf[nb][0];
        la.out_dy = buf[nb][1];
        la.out_dz = buf[nb][2];
        la.H = H;
        la.W = W;
        la.iters = it;
        la.lambda = p->lap_lambda;
        la.out_aos = nullptr;
        remaining -= it;
        if (launch_laplacian(la, lr, s) != cudaSuccess) return PL3D_ERR_CUDA;
        cur = nb;
        first = false;
    } while (remaining > 0);

    // Normals, bilateral, mask and groups in one launch.
    float c_scale = 1.f, a_norm = 0.f;
    bilateral_scales(p->bil_sigma_len, p->bil_sigma_ang, p->bil_iters, &c_scale, &a_norm);
    BilArgs ba;
    ba.points = points;
    ba.dx = buf[cur][0];
    ba.dy = buf[cur][1];
    ba.dz = buf[cur][2];
    ba.carry_in = nullptr;
    ba.carry_out = nullptr;
    ba.out_mask = out_mask;
    ba.out_normals = out_normals;
    ba.out_groups = groups;
    ba.out_labels = out_labels;
    ba.H = H;
    ba.W = W;
    ba.iters = p->bil_iters;
    ba.c_scale = c_scale;
    ba.a_norm = a_norm;
    ba.max_offset_scaled = p->max_offset > 0.f ? p->max_offset * c_scale : 0.f;
    ba.sizes = p->min_triangles > 0 ? sizes : nullptr;
    ba.max_edge2 = p->max_edge > 0.f ? p->max_edge * p->max_edge : INFINITY;
    ba.min_dot = p->min_dot;
    ba.nd = nd;
    if (launch_bilateral(ba, br, true, true, s) != cudaSuccess) return PL3D_ERR_CUDA;

    // Planar segments across tile borders; the bilateral pass zeroed the segment sizes.
    LabelArgs lb;
    lb.groups = groups;
    lb.labels = out_labels;
    lb.sizes = p->min_triangles > 0 ? sizes : nullptr;
    lb.points = points;
    lb.dx = buf[cur][0];
    lb.dy = buf[cur][1];
    lb.dz = buf[cur][2];
    lb.H = H;
    lb.W = W;
    lb.tile_h = kBilTileH;
    lb.tile_w = kBilTileW;
    lb.max_offset = p->max_offset;
    lb.min_triangles = p->min_triangles;
    lb.nd = nd;
    if (launch_label_merge(lb, s) != cudaSuccess) return PL3D_ERR_CUDA;
    if (launch_label_flatten(lb, s) != cudaSuccess) return PL3D_ERR_CUDA;
    if (p->min_triangles > 0 && launch_label_filter(lb, s) != cudaSuccess) return PL3D_ERR_CUDA;
    return PL3D_OK;
}

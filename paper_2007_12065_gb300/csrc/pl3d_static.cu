// pl3d_static.cu -- pl3d_extract_planes_static: the whole path without any allocation.
//
// Who needs it: code that must not allocate device memory after start-up -- a real-time
// sensor loop that has to avoid the device-wide synchronisation cudaMalloc/cudaFree can
// cause, a process whose memory budget was fixed when it started, or a caller with no
// context object to keep (plugins that get a stream and buffers per call). Such a caller
// passes its inputs and outputs; the scratch the path needs (point displacements, groups,
// segment sizes, the grid-barrier and error words) lives in the file-scope device array below
// instead of in a context.
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
// the caller. Nothing in it needs clearing between calls that succeed: every scratch value is
// written before it is read within a call, and the barrier words return to their starting state
// at the end of each call (the array starts zeroed when the library's device code loads). A
// bounded device wait that gives up (grid barrier or TMA, 1 s) leaves the error word set and the
// barrier's arrival count off; pl3d_static_sync reads the error word after the stream's work,
// and when it is set clears it and the barrier words (plain copies and a memset into the same
// array: still no allocation) and reports PL3D_ERR_TIMEOUT.
#include <float.h>
#include <math.h>

#include <mutex>

#include "pl3d_internal.cuh"

using namespace pl3d;

namespace {

constexpr size_t kMaxPoints = PL3D_STATIC_MAX_POINTS;
constexpr size_t kMaxTri = 2 * kMaxPoints;                       // 2(H-1)(W-1) < 2 H W
constexpr size_t kDispBytes = 6 * kMaxPoints * sizeof(float);    // displacement ping-pong, AoS
constexpr size_t kGroupBytes = (kMaxTri + 255) / 256 * 256;
constexpr size_t kSizeBytes = kMaxTri * sizeof(int32_t);
constexpr size_t kCtlBytes = 256;                                // barrier [2], error word, pad,
                                                                 // lap1 task counter [2]
constexpr size_t kScratchBytes = kDispBytes + kGroupBytes + kSizeBytes + kCtlBytes;

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
        if (prop.major != 10 || prop.minor != 3 || !prop.cooperativeLaunch) {
            s.status = PL3D_ERR_UNSUPPORTED;
        } else if (cudaGetSymbolAddress((void**)&s.scratch, g_static_scratch) != cudaSuccess) {
            cudaGetLastError();
            return PL3D_ERR_CUDA;
        } else if (frame_configure() != cudaSuccess) {
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

constexpr size_t kCtlOffset = kDispBytes + kGroupBytes + kSizeBytes;

}  // namespace

namespace pl3d {

// Device address of the allocation-free path's control words (barrier [2], error word, pad) on
// the current device, after the same once-per-device set-up as the entry point.
int static_control_words(unsigned** ctl) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    unsigned char* scratch = nullptr;
    const int rc = setup_device(dev, &scratch);
    if (rc != PL3D_OK) return rc;
    *ctl = reinterpret_cast<unsigned*>(scratch + kCtlOffset);
    return PL3D_OK;
}

}  // namespace pl3d

extern "C" size_t pl3d_static_scratch_bytes(void) { return kScratchBytes; }

extern "C" int pl3d_static_sync(void* stream) {
    unsigned* ctl = nullptr;
    int rc = static_control_words(&ctl);
    if (rc != PL3D_OK) return rc;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PL3D_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return PL3D_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, ctl + 2, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PL3D_ERR_CUDA;
    if (err == 0) return PL3D_OK;
    // a wait gave up: the affected calls' results are void; the control words start over
    if (cudaMemsetAsync(ctl, 0, 4 * sizeof(unsigned), (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return PL3D_ERR_CUDA;
    return PL3D_ERR_TIMEOUT;
}

extern "C" int pl3d_extract_planes_static(const float* points, int H, int W, const pl3d_params* p,
                                          const float* nd_host, int K, uint8_t* out_mask, float* out_normals,
                                          int32_t* out_labels, void* stream) {
    if (!points || !nd_host || !out_mask || !out_normals || !out_labels) return PL3D_ERR_INVALID_ARG;
    int rc = pl3d_validate(p, H, W, nd_host, K);
    if (rc != PL3D_OK) return rc;
    if (p->flags & PL3D_FLAG_SEED_PTP) return PL3D_ERR_UNSUPPORTED;   // host-assisted: needs a context
    if ((size_t)H * (size_t)W > kMaxPoints) return PL3D_ERR_INVALID_ARG;
    if (bilateral_passes(p, Tuning{0, 0, 0}) > 1) return PL3D_ERR_INVALID_ARG;   // would need the carry buffers
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    unsigned char* scratch = nullptr;
    if ((rc = setup_device(dev, &scratch)) != PL3D_OK) return rc;

    FrameScratch sc;
    sc.disp[0] = reinterpret_cast<float*>(scratch);
    sc.disp[1] = sc.disp[0] + 3 * kMaxPoints;
    sc.carry[0] = sc.carry[1] = nullptr;
    sc.groups = scratch + kDispBytes;
    sc.sizes = reinterpret_cast<int32_t*>(scratch + kDispBytes + kGroupBytes);
    unsigned* ctl = reinterpret_cast<unsigned*>(scratch + kCtlOffset);
    sc.barrier = ctl;
    sc.error = reinterpret_cast<int*>(ctl + 2);
    sc.phase_ns = nullptr;
    sc.lap1_sched = ctl + 4;
    sc.border = nullptr;   // the tile borders joined by the merge phase (no counters in the fixed scratch)
    sc.cap_border = 0;
    return frame_launch(sc, points, H, W, p, nd_host, K, out_mask, out_normals, out_labels, nullptr, nullptr,
                        Tuning{0, 0, 0}, (cudaStream_t)stream);
}

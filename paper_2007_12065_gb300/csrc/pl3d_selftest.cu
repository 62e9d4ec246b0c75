// pl3d_selftest.cu -- pl3d_selftest_wait_timeout: makes one of the library's bounded device waits
// run out on purpose, so that the error path (device error word -> PL3D_ERR_TIMEOUT -> control
// words reset) can be checked on a GPU without a fault, a trap or an unbounded wait.
//
// The kernel uses the same wait primitives as the path's kernels (sync.cuh), with the limit
// passed as a kernel argument:
//   kind 1  grid barrier: a cooperative grid of two CTAs in which the last CTA returns without
//           arriving; the other one waits for it until the limit, sets the barrier-timeout bit
//           and returns (the barrier's arrival count is left at one, as after a real timeout);
//   kind 2  mbarrier: one CTA initialises an mbarrier that nothing arms and waits on its first
//           phase until the limit (twice, as a real TMA wait does for copies in flight), sets the
//           TMA-timeout bit and returns. No copy is issued.
#include "pl3d_ctx.cuh"
#include "sync.cuh"

using namespace pl3d;

namespace {

constexpr int kKindBarrier = 1;
constexpr int kKindMbarrier = 2;

__global__ void wait_selftest_kernel(unsigned* bar, int* err, int kind, unsigned long long limit_ns) {
    if (kind == kKindBarrier) {
        if (blockIdx.x == gridDim.x - 1) return;   // leaves without arriving at the barrier
        grid_barrier(bar, err, limit_ns);
    } else if (kind == kKindMbarrier && blockIdx.x == 0) {
        __shared__ __align__(8) uint64_t mb;
        if (threadIdx.x == 0) mbar_init(&mb, 1);
        __syncthreads();
        if (threadIdx.x == 0) mbar_wait_bounded(&mb, 0u, err, limit_ns);
        __syncthreads();
    }
}

int launch_selftest(unsigned* ctl, int kind, int64_t limit_ns, cudaStream_t s) {
    unsigned* bar = ctl;
    int* err = reinterpret_cast<int*>(ctl + 2);
    unsigned long long lim = (unsigned long long)limit_ns;
    void* args[4] = {&bar, &err, &kind, &lim};
    if (cudaLaunchCooperativeKernel((const void*)wait_selftest_kernel, dim3(2), dim3(32), args, 0, s) != cudaSuccess) {
        cudaGetLastError();
        return PL3D_ERR_CUDA;
    }
    return PL3D_OK;
}

}  // namespace

extern "C" int pl3d_selftest_wait_timeout(pl3d_ctx* ctx, int kind, int64_t limit_ns, void* stream) {
    if (kind != kKindBarrier && kind != kKindMbarrier) return PL3D_ERR_INVALID_ARG;
    if (limit_ns < 100000 || limit_ns > 10000000000LL) return PL3D_ERR_INVALID_ARG;
    if (!ctx) {
        unsigned* ctl = nullptr;
        const int rc = static_control_words(&ctl);
        if (rc != PL3D_OK) return rc;
        return launch_selftest(ctl, kind, limit_ns, (cudaStream_t)stream);
    }
    ctxutil::DeviceGuard g(ctx->device);
    if (!g.ok) return PL3D_ERR_CUDA;
    const int rc = launch_selftest(ctx->ctl, kind, limit_ns, (cudaStream_t)stream);
    if (rc == PL3D_OK) ctx->launches += 1;
    return rc;
}

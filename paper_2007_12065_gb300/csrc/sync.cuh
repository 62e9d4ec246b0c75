// sync.cuh -- TMA tile loads, mbarriers and a grid-wide barrier, all with bounded waits.
//
// Every wait here gives up after limit_ns of %globaltimer time (kWaitLimitNs unless the caller
// passes a shorter limit, as the wait self-test kernel does) and an iteration cap, records the
// reason in the frame's device error word and returns, so a fault elsewhere surfaces as
// PL3D_ERR_TIMEOUT on the host instead of a hung GPU.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pl3d {

constexpr uint64_t kWaitLimitNs = 1000000000ull;   // 1 s
constexpr int kErrTmaTimeout = 1;                  // bits of the device error word
constexpr int kErrBarrierTimeout = 2;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders earlier generic-proxy accesses (this CTA's shared memory; global memory written by
// any CTA before a grid barrier) before later async-proxy (TMA) accesses.
// Orders this CTA's earlier generic-proxy shared-memory accesses (made visible to the issuing
// thread by a __syncthreads) before its later async-proxy (TMA) writes to shared memory.
__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_all() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Makes a tensor map that the host copied into global memory before the launch visible to the
// tensor-map proxy of this thread (issued before the thread's first TMA through that map; the
// map was written by a host-initiated copy, hence system scope).
__device__ __forceinline__ void tensormap_acquire(const void* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Tests for the completion of phase `parity`; a thread whose phase is still pending is suspended
// in hardware for up to kSuspendNs (or until the phase completes) instead of spinning.
constexpr uint32_t kSuspendNs = 100000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// 2-D tiled TMA load of a box at element coordinates (x, y) into shared memory; completion is
// counted in bytes on `bar`. x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Waits for the phase `parity` of `bar` to complete. On timeout it records the error, waits
// once more (bounded) for the copies still in flight, and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* err,
                                                  uint64_t limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const uint64_t t0 = global_ns();
        for (uint32_t i = 0; i < (1u << 24); ++i) {
            if (mbar_try_wait(bar, parity)) return attempt == 0;
            if (global_ns() - t0 > limit_ns) break;
        }
        if (attempt == 0) atomicOr(err, kErrTmaTimeout);
    }
    return false;
}

// Acquire load, acquire-release add and release add at GPU scope (PTX memory consistency model).
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a co-resident (cooperatively launched) grid. bar[0] counts arrivals,
// bar[1] is the generation. Thread 0 of each CTA arrives with an acquire-release add, which
// publishes the writes its CTA made before the __syncthreads (cumulativity) and, for the last
// arriver, acquires everyone else's; the last arriver resets the count and opens the barrier
// with a release add on the generation, which the others wait for with acquire loads. Global
// writes made before the barrier are visible to every thread of the grid after it.
__device__ __forceinline__ void grid_barrier(unsigned* bar, int* err, uint64_t limit_ns = kWaitLimitNs) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
        const unsigned g = ld_acquire_gpu(bar + 1);   // cannot advance before this CTA arrives
        if (atom_add_acq_rel_gpu(bar, 1u) + 1u == nblocks) {
            *reinterpret_cast<volatile unsigned*>(bar) = 0u;   // ordered before the release below
            red_release_gpu_add(bar + 1, 1u);
        } else {
            const uint64_t t0 = global_ns();
            for (uint32_t i = 1; ld_acquire_gpu(bar + 1) == g; ++i) {
                if ((i & 63u) == 0u && global_ns() - t0 > limit_ns) {
                    atomicOr(err, kErrBarrierTimeout);
                    break;
                }
                __nanosleep(16);
            }
        }
    }
    __syncthreads();
}

}  // namespace pl3d

// uf.cuh -- lock-free union-find over an int32 parent array (shared or global memory).
//
// Every parent pointer points to a smaller-or-equal index, and a root is only linked below a
// smaller root, with a compare-and-swap on the larger root. So each component ends with its
// smallest index as root, whatever order the unions run in, and the result is deterministic.
// Finding halves the path as it walks: each visited node is pointed at its grandparent, an
// ancestor, so concurrent walks and links stay valid. Walks that run after all unions have
// finished use the read-only form.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pl3d {

__device__ __forceinline__ int uf_find(int32_t* L, int x) {
    volatile int32_t* vl = L;
    while (true) {
        const int p = vl[x];
        if (p == x) return x;
        const int gp = vl[p];
        if (gp == p) return p;
        vl[x] = gp;
        x = gp;
    }
}

__device__ __forceinline__ void uf_unite(int32_t* L, int a, int b) {
    while (true) {
        a = uf_find(L, a);
        b = uf_find(L, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(L + b, b, a);
        if (old == b) return;
        b = old;   // b stopped being a root meanwhile; continue from its new parent
    }
}

// Root of x when no union runs concurrently (reads only).
__device__ __forceinline__ int uf_root(const int32_t* L, int x) {
    const volatile int32_t* vl = L;
    int p = vl[x];
    while (p != x) {
        x = p;
        p = vl[x];
    }
    return x;
}

}  // namespace pl3d

// f32x2.cuh -- packed pairs of FP32 values and Blackwell's paired FP32 instructions
// (PTX add/sub/mul/fma.rn.f32x2): one instruction, two independent IEEE round-to-nearest
// results, each bit-identical to the scalar instruction on its half.
#pragma once

#include <cuda_runtime.h>

namespace pl3d {

typedef unsigned long long f2;   // {lo, hi}

__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ f2 bc(float v) { return pk(v, v); }

__device__ __forceinline__ void upk(f2 v, float& lo, float& hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }

__device__ __forceinline__ float lo_of(f2 v) {
    float lo, hi;
    upk(v, lo, hi);
    return lo;
}

__device__ __forceinline__ float hi_of(f2 v) {
    float lo, hi;
    upk(v, lo, hi);
    return hi;
}

__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

}  // namespace pl3d

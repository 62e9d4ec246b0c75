// df32.cuh -- error-free float transformations used to keep the smoothed geometry accurate.
//
// A smoothed point is carried as its FP32 input position v0 plus an FP32 displacement d
// (v = v0 + d, never rounded to one float while the path runs). Differences between points
// and the cross products of triangle edges are then formed as unevaluated float pairs
// (hi + lo) with Knuth's TwoSum and the FMA-based TwoProduct, so sliver triangles (edges of
// tens of metres with millimetre heights at depth discontinuities) keep their normals to
// about 1e-7 rad instead of inheriting the ~1e-7 relative rounding of an FP32 coordinate.
// The _rn intrinsics keep the compiler from contracting or reassociating these steps.
#pragma once

#include <cuda_runtime.h>

namespace pl3d {

struct F2 {
    float h, l;
};

// s + e == a + b exactly (Knuth, TAOCP vol. 2, 4.2.2).
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// p + e == a * b exactly (one FMA recovers the rounding error of the product).
__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// (b0 + bd) - (a0 + ad) as a float pair: the two differences are exact, their sum keeps
// its rounding error in lo.
__device__ __forceinline__ F2 pair_diff(float a0, float ad, float b0, float bd) {
    const F2 s = two_sum(b0, -a0);
    const F2 t = two_sum(bd, -ad);
    const F2 u = two_sum(s.h, t.h);
    const float lo = __fadd_rn(u.l, __fadd_rn(s.l, t.l));
    return two_sum(u.h, lo);
}

// a * b for float pairs, dropping a.l * b.l (relative size 2^-48).
__device__ __forceinline__ F2 pair_mul(F2 a, F2 b) {
    F2 p = two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return p;
}

// a - b for float pairs, rounded once to float.
__device__ __forceinline__ float pair_sub_round(F2 a, F2 b) {
    const F2 s = two_sum(a.h, -b.h);
    return __fadd_rn(s.h, __fadd_rn(s.l, __fsub_rn(a.l, b.l)));
}

// Square of a float pair, rounded once to float.
__device__ __forceinline__ float pair_sq_round(F2 a) {
    const F2 p = two_prod(a.h, a.h);
    return __fadd_rn(p.h, __fmaf_rn(2.0f * a.h, a.l, p.l));
}

}  // namespace pl3d

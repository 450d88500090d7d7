// FP32-pair ("double-float") arithmetic.
//
// A value is carried as hi + lo with |lo| <= ulp(hi)/2.  GB300 runs FP32 FMAs
// about 60x faster than FP64 ones, so FP64-accuracy dot products with many
// terms are done on pairs: each product's rounding error is recovered
// exactly with an FMA (Dekker's product), the running sum's with Knuth's
// TwoSum, and the errors are accumulated apart from the sum (the
// Ogita-Rump-Oishi Dot2 scheme, extended to pair inputs by the two cross
// terms).  Intrinsics with explicit rounding keep the compiler from fusing or
// reassociating the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace smm {

__device__ __forceinline__ void df_split(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

__device__ __forceinline__ float2 df_make(double v) {
    float2 r;
    df_split(v, r.x, r.y);
    return r;
}

// (s, c) += (ah + al) * (xh + xl), the al * xl term dropped (2^-48 relative)
__device__ __forceinline__ void df_acc(float& s, float& c, float ah, float al, float xh, float xl) {
    const float ph = __fmul_rn(ah, xh);
    float t = __fmaf_rn(ah, xh, -ph);  // exact rounding error of ah * xh
    t = __fmaf_rn(ah, xl, t);
    t = __fmaf_rn(al, xh, t);
    const float sn = __fadd_rn(s, ph);  // TwoSum(s, ph)
    const float bp = __fsub_rn(sn, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bp)), __fsub_rn(ph, bp));
    c = __fadd_rn(c, __fadd_rn(err, t));
    s = sn;
}

// (s, c) += (vh + vl)
__device__ __forceinline__ void df_add(float& s, float& c, float vh, float vl) {
    const float sn = __fadd_rn(s, vh);
    const float bp = __fsub_rn(sn, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bp)), __fsub_rn(vh, bp));
    c = __fadd_rn(c, __fadd_rn(err, vl));
    s = sn;
}

// renormalize (s, c) into a pair with |lo| <= ulp(hi)/2 (c small next to s)
__device__ __forceinline__ float2 df_norm(float s, float c) {
    const float h = __fadd_rn(s, c);
    return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

__device__ __forceinline__ double df_to_double(float s, float c) { return (double)s + (double)c; }

}  // namespace smm

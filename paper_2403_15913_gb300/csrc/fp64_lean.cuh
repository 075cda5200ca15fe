// FP64 helpers that spend few FP64 issue slots.  On GB300 a warp FP64
// instruction occupies its sub-partition's FP64 unit for 64 cycles whatever
// the number of active lanes, while integer and FP32 instructions issue at
// full rate, so elementwise kernels with divisions, square roots and format
// conversions are bound by the FP64 unit long before HBM.  These helpers move
// what they can to the integer and FP32 units:
//
//  * f32_of / f64_of: double <-> float of a positive normal number by the
//    IEEE-754 bit layout (exponent rebiased by 1023 - 127 = 896, mantissa
//    truncated to 23 bits / widened with zeros): integer shifts and adds.
//    Valid in the range (kLeanLo, kLeanHi), where both formats are normal.
//  * rcp_pos: 1/d for d > 0.  Seed y0 = the FP32 reciprocal of f32_of(d)
//    (relative error e0 below 2^-22), then one third-order Newton-Householder
//    step for the reciprocal: with e = 1 - d y0, 1/d = y0 / (1 - e) =
//    y0 (1 + e + e^2 + O(e^3)), truncation below 2^-66 -- three FP64 FMAs.
//    Outside the range, the IEEE division.
#pragma once
#include <cuda_runtime.h>

namespace kktgb {

constexpr long long kLeanLo = 0x39b4484bfeebc2a0LL;   // bits of 1e-30
constexpr long long kLeanHi = 0x46293e5939a08ceaLL;   // bits of 1e30

__device__ __forceinline__ bool lean_range(double d) {
    const long long b = __double_as_longlong(d);
    return b > kLeanLo && b < kLeanHi;
}

__device__ __forceinline__ float f32_of(double d) {
    return __int_as_float((int)((__double_as_longlong(d) >> 29) - (896LL << 23)));
}

__device__ __forceinline__ double f64_of(float y) {
    return __longlong_as_double(((long long)__float_as_int(y) << 29) + (896LL << 52));
}

__device__ __forceinline__ double rcp_pos(double d) {
    if (!lean_range(d)) return 1.0 / d;
    const double y0 = f64_of(__frcp_rn(f32_of(d)));
    const double e = fma(-d, y0, 1.0);
    return fma(fma(e, e, e), y0, y0);
}

}  // namespace kktgb

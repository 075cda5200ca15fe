// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, carrying ~48 bits of
// significand.  On GB300 the FP32 pipe issues 64x the FP64 rate (a warp FP64
// FMA occupies a sub-partition's FP64 unit for 64 cycles), so a double-float
// fused multiply-add of ~15 FP32 instructions is still ~4x faster than a
// native FP64 one.  The factor kernels instantiated on this type produce a
// factor with unit roundoff ~2^-47 that preconditions the FP64 refinement.
//
// Built from the error-free transformations of the literature:
//   TwoSum (Knuth, TAOCP vol. 2): s = fl(a + b) and the exact error e, with
//     a + b = s + e, for any a, b;
//   FastTwoSum (Dekker 1971): the same in three operations when |a| >= |b|;
//   TwoProduct with a fused multiply-add: p = fl(a b), e = fma(a, b, -p)
//     exact (a b = p + e).
// The multiply-add below adds the cross products and the low parts without
// compensation (the "sloppy" variants of double-double arithmetic): its error
// is a few units of 2^-48 relative to the magnitude of the terms, the
// normwise error a Cholesky factorisation is analysed with.
#pragma once
#include <cuda_runtime.h>

namespace kktgb {

struct df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ df64(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
    const float s = a + b;
    return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
    float s1, s2, t1, t2;
    two_sum(x.hi, y.hi, s1, s2);
    two_sum(x.lo, y.lo, t1, t2);
    s2 += t1;
    df64 u = fast_two_sum(s1, s2);
    return fast_two_sum(u.hi, u.lo + t2);
}

__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
    const float p = x.hi * y.hi;
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

// a b + c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
    const float p = a.hi * b.hi;
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(p, c.hi, s, t);
    t += e + c.lo;
    return fast_two_sum(s, t);
}

__device__ __forceinline__ df64& operator+=(df64& x, df64 y) { return x = x + y; }
__device__ __forceinline__ df64& operator-=(df64& x, df64 y) { return x = x - y; }
__device__ __forceinline__ df64& operator*=(df64& x, df64 y) { return x = x * y; }

__device__ __forceinline__ bool operator>(df64 x, double v) {
    const df64 y(v);
    return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo);
}

__device__ __forceinline__ bool isfinite(df64 x) { return ::isfinite(x.hi) && ::isfinite(x.lo); }

__device__ __forceinline__ bool pivot_ok(df64 d) { return d > 0.0 && isfinite(d); }

// 1/sqrt(d): FP32 seed (the library reciprocal square root), then two Newton
// steps y <- y + y (1 - d y^2) / 2 in double-float arithmetic, each roughly
// doubling the correct bits (~22 -> ~44 -> ~48).
__device__ __forceinline__ df64 pivot_rsqrt(df64 d) {
    df64 y(rsqrtf(d.hi), 0.0f);
    const df64 half(0.5f, 0.0f), one(1.0f, 0.0f);
    for (int it = 0; it < 2; ++it) {
        const df64 r = one - d * (y * y);
        y = fma(y * half, r, y);
    }
    return y;
}

__device__ __forceinline__ df64 __shfl_sync(unsigned mask, df64 v, int lane) {
    return df64(::__shfl_sync(mask, v.hi, lane), ::__shfl_sync(mask, v.lo, lane));
}

__device__ __forceinline__ df64 __shfl_down_sync(unsigned mask, df64 v, unsigned delta) {
    return df64(::__shfl_down_sync(mask, v.hi, delta), ::__shfl_down_sync(mask, v.lo, delta));
}

__device__ __forceinline__ df64 __shfl_xor_sync(unsigned mask, df64 v, int lanemask) {
    return df64(::__shfl_xor_sync(mask, v.hi, lanemask), ::__shfl_xor_sync(mask, v.lo, lanemask));
}

__device__ __forceinline__ df64 __ldcg(const df64* p) {
    const float2 f = ::__ldcg(reinterpret_cast<const float2*>(p));
    return df64(f.x, f.y);
}

// atomic x += v by compare-and-swap of the 8-byte pair
__device__ __forceinline__ df64 atomicAdd(df64* addr, df64 v) {
    unsigned long long* a = reinterpret_cast<unsigned long long*>(addr);
    unsigned long long old = *a, assumed;
    do {
        assumed = old;
        df64 cur;
        memcpy(&cur, &assumed, sizeof(cur));
        const df64 nv = cur + v;
        unsigned long long bits;
        memcpy(&bits, &nv, sizeof(bits));
        old = atomicCAS(a, assumed, bits);
    } while (old != assumed);
    df64 prev;
    memcpy(&prev, &old, sizeof(prev));
    return prev;
}

}  // namespace kktgb

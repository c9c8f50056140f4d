// Double-float ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two float32 numbers with |lo| <= ulp(hi)/2, giving about 48
// significant bits on the float32 pipes.  GB300 issues float32 FMAs at 64x its
// float64 rate, so float64-accuracy FFTs run faster this way.  Error-free
// transformations: Knuth's two-sum, Dekker's fast two-sum, and the
// FMA-based two-product (a*b - fl(a*b) computed exactly by one fmaf).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace nufft45 {

struct dd {
    float hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of a double (exact for |x| in the float range to ~2^-48 relative)
    __host__ __device__ constexpr dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ constexpr dd(int x) : hi((float)x), lo(0.f) {}
};

__host__ __device__ __forceinline__ dd dd_fast_two_sum(float a, float b) {
    const float s = a + b;
    return dd(s, b - (s - a));
}

__host__ __device__ __forceinline__ dd dd_two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    return dd(s, (a - (s - v)) + (b - v));
}

__host__ __device__ __forceinline__ dd operator+(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__host__ __device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dd_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ dd& operator+=(dd& a, dd b) { a = a + b; return a; }
__host__ __device__ __forceinline__ dd& operator-=(dd& a, dd b) { a = a - b; return a; }
__host__ __device__ __forceinline__ dd& operator*=(dd& a, dd b) { a = a * b; return a; }

__device__ __forceinline__ double dd_to_double(dd a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dd dd_from_double(double x) {
    const float h = __double2float_rn(x);
    return dd(h, __double2float_rn(x - (double)h));
}

// complex double-float: the layout of float4 (re.hi, re.lo, im.hi, im.lo)
struct __align__(16) cdd {
    dd x, y;
};
template <> struct C2<dd> { using type = cdd; };

template <> __device__ __forceinline__ cdd ldg<cdd>(const cdd* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    cdd r;
    r.x = dd(v.x, v.y);
    r.y = dd(v.z, v.w);
    return r;
}
template <> __device__ __forceinline__ dd ldg<dd>(const dd* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return dd(v.x, v.y);
}

}  // namespace nufft45

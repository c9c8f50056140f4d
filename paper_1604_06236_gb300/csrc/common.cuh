// Shared device helpers for the nufft45 library: complex arithmetic on
// interleaved (re, im) pairs, exact fixed-point phases, the spreading kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nufft45 {

// ---- complex arithmetic on float2 / double2 --------------------------------
template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <typename T> using c2 = typename C2<T>::type;

template <typename T> __host__ __device__ __forceinline__ c2<T> mk(T re, T im) { c2<T> r; r.x = re; r.y = im; return r; }
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
    V r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
// multiply by +j (dir=+1) or -j (dir=-1)
template <typename V> __host__ __device__ __forceinline__ V cmulj(V a, int dir) {
    V r; if (dir > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; } return r;
}
template <typename V> __host__ __device__ __forceinline__ V cfma(V acc, V a, V b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

// Programmatic dependent launch: the library launches every kernel as a
// dependent of the previous one in its stream, so a kernel's launch and CTA
// scheduling overlap its predecessor's tail.  Every kernel therefore starts
// with pdl_wait(), which returns once the predecessor grid has completed and
// its memory operations are visible (at once for an ordinary launch), and
// then allows its own successor to be scheduled with pdl_trigger().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// read-only-path load (the double-float types specialise it)
template <typename X> __device__ __forceinline__ X ldg(const X* p) { return __ldg(p); }

template <typename To, typename From> __host__ __device__ __forceinline__ c2<To> ccast(From a) {
    return mk<To>((To)a.x, (To)a.y);
}

// ---- exact phases ----------------------------------------------------------
// A node t in [0,1) is carried as T = t * 2^64 (uint64).  e^{j 2 pi m t} then
// has the exact turn count m*T mod 2^64, so only the final sin/cos rounds.
__device__ __forceinline__ double turns_of(uint64_t ph) {
    return (double)(int64_t)ph * 5.42101086242752217003726400434970855712890625e-20;  // 2^-64, in [-1/2, 1/2)
}
// e^{sign * j 2 pi ph / 2^64} in double
__device__ __forceinline__ double2 cis_turns(uint64_t ph, int sign) {
    double s, c;
    sincospi(2.0 * turns_of(ph), &s, &c);
    return make_double2(c, sign >= 0 ? s : -s);
}

// ---- "exponential of semicircle" spreading kernel ---------------------------
// phi(z) = exp(beta (sqrt(1 - z^2) - 1)) for |z| < 1, 0 otherwise, with z =
// 2 d / w for a grid offset d and an even width w (Barnett, Magland and
// af Klinteberg, SIAM J. Sci. Comput. 2019).
template <typename T> __device__ __forceinline__ T es_kernel(T d, T two_over_w, T beta) {
    T z = d * two_over_w;
    T a = (T)1 - z * z;
    return a > (T)0 ? exp(beta * (sqrt(a) - (T)1)) : (T)0;
}
template <> __device__ __forceinline__ float es_kernel<float>(float d, float two_over_w, float beta) {
    float z = d * two_over_w;
    float a = 1.0f - z * z;
    return a > 0.0f ? expf(beta * (sqrtf(a) - 1.0f)) : 0.0f;
}

__host__ __device__ __forceinline__ int64_t imod(int64_t a, int64_t n) { a %= n; return a < 0 ? a + n : a; }

}  // namespace nufft45

#define NUFFT_CUDA_TRY(expr)                                  \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return ::nufft45::cuda_fail(_e, #expr, __FILE__, __LINE__); \
    } while (0)

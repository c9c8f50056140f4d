// e^{j 2 pi T / 2^64} for an exact 64-bit turn count T with few float64
// operations (GB300 issues float64 at 1/64 of its float32 rate): the top 12
// bits of T index a table of e^{j 2 pi i / 4096}, and the remaining angle
// theta = 2 pi (T mod 2^52) / 2^64 < 2 pi / 4096 enters through its Taylor
// series, cos to theta^4 and sin to theta^5 (truncation below 3e-20).  One
// complex product joins them: about 2 ulp, against ~1 ulp for sincospi, at
// less than half its cost.
//
// The tables (this one and exp_t's) are per-translation-unit __device__
// arrays; cis_table_ensure() fills them on the current device (once per
// device, from long double host trigonometry and exp2) and must run before
// the first launch that reads them.
#pragma once
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.h"

namespace nufft45 {

static __device__ double2 g_cis_table[4096];
static __device__ double g_exp2_table[64];   // 2^(j/64), j < 64

// e^x for |x| < 700 in float64, by P. T. P. Tang's table-driven method
// ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989): x = (64 m + j) ln2/64 + r,
// |r| <= ln2/128, the reduction done with an FMA against ln2/64 split into a
// float64 head and its (tiny) remainder, so that k ln2/64 enters without
// rounding; e^x = 2^m 2^(j/64) (1 + p), p = e^r - 1 by its Taylor series to
// r^6 (truncation below |r|^7/5040 < 3e-20).  About 3 ulp; 12 float64
// operations against the ~2x more of a general-purpose exponential.
__device__ __forceinline__ double exp_t(double x) {
    const double kd = rint(x * 92.33248261689366);                  // 64 / ln2
    double r = fma(-kd, 0x1.62e42fefa39efp-7, x);                    // ln2/64, head
    r = fma(-kd, 0x1.abc9e3b39803fp-62, r);                          // ln2/64 - head
    const double p =
        r * fma(r, fma(r, fma(r, fma(r, fma(r, 1.0 / 720.0, 1.0 / 120.0), 1.0 / 24.0), 1.0 / 6.0), 0.5), 1.0);
    const int k = (int)kd;
    const double t = g_exp2_table[k & 63];
    const double sc = __longlong_as_double((long long)((k >> 6) + 1023) << 52);   // 2^m
    return fma(t, p, t) * sc;
}

__device__ __forceinline__ double2 cis_turns_t(uint64_t T, int sign) {
    const double2 t = g_cis_table[T >> 52];
    // 2 pi / 2^64
    const double th = (double)(T & ((1ull << 52) - 1)) * 3.4061215800865545e-19;
    const double t2 = th * th;
    const double c = fma(t2, fma(t2, 1.0 / 24.0, -0.5), 1.0);
    const double s = th * fma(t2, fma(t2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
    double2 r;
    r.x = fma(t.x, c, -t.y * s);
    r.y = fma(t.x, s, t.y * c);
    if (sign < 0) r.y = -r.y;
    return r;
}

[[maybe_unused]] static nufft_status cis_table_ensure() {
    static std::atomic<bool> done[64];
    static std::mutex mu;
    int dev = 0;
    NUFFT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(NUFFT_ERR_ARG, "device %d out of range", dev);
    if (done[dev].load(std::memory_order_acquire)) return NUFFT_OK;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev].load(std::memory_order_relaxed)) return NUFFT_OK;
    std::vector<double2> h(4096);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int i = 0; i < 4096; ++i) {
        const long double a = two_pi * (long double)i / 4096.0L;
        h[i] = make_double2((double)cosl(a), (double)sinl(a));
    }
    NUFFT_CUDA_TRY(cudaMemcpyToSymbol(g_cis_table, h.data(), sizeof(double2) * h.size()));
    std::vector<double> e2(64);
    for (int j = 0; j < 64; ++j) e2[j] = (double)exp2l((long double)j / 64.0L);
    NUFFT_CUDA_TRY(cudaMemcpyToSymbol(g_exp2_table, e2.data(), sizeof(double) * e2.size()));
    done[dev].store(true, std::memory_order_release);
    return NUFFT_OK;
}

}  // namespace nufft45

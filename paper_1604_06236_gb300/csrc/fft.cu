// Stockham autosort FFT for any length, staged through shared memory.
//
// A length n with prime factors in {2,3,5,7} is split into passes of
// composite radix R_i (prod R_i = n, R_i <= 512 for complex64 and <= 256 for
// complex128).  Each pass reads and writes the array once, fully coalesced:
// a CTA loads C butterflies (C consecutive j, each with R inputs of stride
// n/R), applies the inter-pass twiddles, performs the C length-R DFTs in
// shared memory with radix-2/3/4/5/7/8 Stockham sub-stages (ping-pong
// buffers), and stores the results in Stockham order, so the final pass leaves
// the transform in natural order.  Lengths with a larger prime factor use
// Bluestein's chirp-z convolution on a smooth length m >= 2n - 1.
#include <atomic>
#include "internal.h"
#include "df.cuh"
#include "fft_p2.cuh"
#include "fft_p2t.cuh"
#include "fft_ddq.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

namespace nufft45 {

namespace {

constexpr int kThreads = 256;

template <typename T> struct FftLimits;
template <> struct FftLimits<float> { static constexpr int kElems = 8192; static constexpr int kLmax = 512; };
template <> struct FftLimits<double> { static constexpr int kElems = 4096; static constexpr int kLmax = 256; };
template <> struct FftLimits<dd> { static constexpr int kElems = 4096; static constexpr int kLmax = 256; };

struct PassArgs {
    int64_t n, nR, Ns, total;  // total = batch * n / R butterflies
    int R, PR, C, nsub;
    int sub[12];
    int in_cfast, out_cfast;
    int shift;
    int64_t mask;
};

template <typename T>
__device__ __forceinline__ c2<T> twiddle(const c2<T>* __restrict__ lo, const c2<T>* __restrict__ hi, int shift,
                                         int64_t mask, int64_t e, int dir) {
    c2<T> w = cmul(ldg(&lo[e & mask]), ldg(&hi[e >> shift]));
    if (dir > 0) w.y = -w.y;
    return w;
}

// ---- small DFTs in registers (dir = -1 forward, +1 inverse) ----------------
template <typename V> __device__ __forceinline__ void dft2(V* v) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
}
template <typename V> __device__ __forceinline__ void dft4(V* v, int dir) {
    V s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    V s13 = cadd(v[1], v[3]), d13 = cmulj(csub(v[1], v[3]), dir);
    v[0] = cadd(s02, s13); v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13); v[3] = csub(d02, d13);
}
template <typename V> __device__ __forceinline__ void dft8(V* v, int dir) {
    using T = decltype(v[0].x);
    const T h = (T)0.70710678118654752440;
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e, dir); dft4(o, dir);
    // W8^1 = h (1 + dir j), W8^2 = dir j, W8^3 = h (-1 + dir j)
    V o1 = cscale(cadd(o[1], cmulj(o[1], dir)), h);
    V o2 = cmulj(o[2], dir);
    V o3 = cscale(csub(cmulj(o[3], dir), o[3]), h);
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
}
template <typename V> __device__ __forceinline__ void dft3(V* v, int dir) {
    using T = decltype(v[0].x);
    const T s3 = (T)0.86602540378443864676;   // sin(2 pi / 3)
    V t1 = cadd(v[1], v[2]);
    V t2 = csub(v[0], cscale(t1, (T)0.5));
    V t3 = cmulj(cscale(csub(v[1], v[2]), s3), dir);
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
}
template <typename V> __device__ __forceinline__ void dft5(V* v, int dir) {
    using T = decltype(v[0].x);
    const T c1 = (T)0.30901699437494742410, c2_ = (T)-0.80901699437494742410;   // cos(2pi/5), cos(4pi/5)
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;    // sin(2pi/5), sin(4pi/5)
    V a0 = v[0];
    V p1 = cadd(v[1], v[4]), m1 = csub(v[1], v[4]);
    V p2 = cadd(v[2], v[3]), m2 = csub(v[2], v[3]);
    V r1 = cadd(a0, cadd(cscale(p1, c1), cscale(p2, c2_)));
    V r2 = cadd(a0, cadd(cscale(p1, c2_), cscale(p2, c1)));
    V i1 = cmulj(cadd(cscale(m1, s1), cscale(m2, s2)), dir);
    V i2 = cmulj(csub(cscale(m1, s2), cscale(m2, s1)), dir);
    v[0] = cadd(a0, cadd(p1, p2));
    v[1] = cadd(r1, i1); v[4] = csub(r1, i1);
    v[2] = cadd(r2, i2); v[3] = csub(r2, i2);
}
// radix 7: direct DFT with W_7 from the length-n twiddle table (7 | n)
template <typename T>
__device__ __forceinline__ void dft7(c2<T>* v, int dir, const c2<T>* lo, const c2<T>* hi, int shift,
                                     int64_t mask, int64_t n) {
    c2<T> w[7];
    for (int q = 0; q < 7; ++q) w[q] = twiddle<T>(lo, hi, shift, mask, (int64_t)q * (n / 7), dir);
    c2<T> out[7];
    for (int m = 0; m < 7; ++m) {
        c2<T> acc = v[0];
        for (int k = 1; k < 7; ++k) acc = cadd(acc, cmul(v[k], w[(m * k) % 7]));
        out[m] = acc;
    }
    for (int m = 0; m < 7; ++m) v[m] = out[m];
}

template <typename T, int r>
__device__ __forceinline__ void substage(const c2<T>* __restrict__ src, c2<T>* __restrict__ dst, int R, int PR,
                                         int C, int Nsub, int dir, const c2<T>* lo, const c2<T>* hi, int shift,
                                         int64_t mask, int64_t n) {
    const int Rr = R / r;
    const int nbf = C * Rr;
    for (int bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
        const int c = bf / Rr, jj = bf - c * Rr;
        const c2<T>* s = src + c * PR;
        c2<T> v[r];
#pragma unroll
        for (int k = 0; k < r; ++k) v[k] = s[jj + k * Rr];
        const int jm = jj % Nsub;
        if (jm != 0) {
            const int64_t step = (int64_t)jm * (n / ((int64_t)Nsub * r));
#pragma unroll
            for (int k = 1; k < r; ++k) v[k] = cmul(v[k], twiddle<T>(lo, hi, shift, mask, step * k, dir));
        }
        if constexpr (r == 2) dft2(v);
        else if constexpr (r == 3) dft3(v, dir);
        else if constexpr (r == 4) dft4(v, dir);
        else if constexpr (r == 5) dft5(v, dir);
        else if constexpr (r == 8) dft8(v, dir);
        else dft7<T>(v, dir, lo, hi, shift, mask, n);
        c2<T>* d = dst + c * PR + (jj / Nsub) * Nsub * r + jm;
#pragma unroll
        for (int m = 0; m < r; ++m) d[m * Nsub] = v[m];
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fft_pass(const c2<T>* in, c2<T>* out,  // may alias (single pass)
                                                       PassArgs a, const c2<T>* __restrict__ lo,
                                                       const c2<T>* __restrict__ hi, int dir) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* s0 = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* s1 = s0 + (size_t)a.C * a.PR;
    const int64_t g0 = (int64_t)blockIdx.x * a.C;
    const int tot = a.C * a.R;
    const int64_t tw_step = a.n / (a.Ns * a.R);
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        int c, k;
        if (a.in_cfast) { c = e % a.C; k = e / a.C; } else { k = e % a.R; c = e / a.R; }
        const int64_t g = g0 + c;
        c2<T> x = mk<T>(0, 0);
        if (g < a.total) {
            const int64_t b = g / a.nR, j = g - b * a.nR;
            x = in[b * a.n + j + (int64_t)k * a.nR];
            const int64_t jm = j % a.Ns;
            if (jm != 0 && k != 0) x = cmul(x, twiddle<T>(lo, hi, a.shift, a.mask, jm * k * tw_step, dir));
        }
        s0[c * a.PR + k] = x;
    }
    __syncthreads();
    c2<T>* src = s0;
    c2<T>* dst = s1;
    int Nsub = 1;
    for (int st = 0; st < a.nsub; ++st) {
        const int r = a.sub[st];
        switch (r) {
            case 2: substage<T, 2>(src, dst, a.R, a.PR, a.C, Nsub, dir, lo, hi, a.shift, a.mask, a.n); break;
            case 3: substage<T, 3>(src, dst, a.R, a.PR, a.C, Nsub, dir, lo, hi, a.shift, a.mask, a.n); break;
            case 4: substage<T, 4>(src, dst, a.R, a.PR, a.C, Nsub, dir, lo, hi, a.shift, a.mask, a.n); break;
            case 5: substage<T, 5>(src, dst, a.R, a.PR, a.C, Nsub, dir, lo, hi, a.shift, a.mask, a.n); break;
            case 7: substage<T, 7>(src, dst, a.R, a.PR, a.C, Nsub, dir, lo, hi, a.shift, a.mask, a.n); break;
            default: substage<T, 8>(src, dst, a.R, a.PR, a.C, Nsub, dir, lo, hi, a.shift, a.mask, a.n); break;
        }
        __syncthreads();
        c2<T>* t = src; src = dst; dst = t;
        Nsub *= r;
    }
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        int c, m;
        if (a.out_cfast) { c = e % a.C; m = e / a.C; } else { m = e % a.R; c = e / a.R; }
        const int64_t g = g0 + c;
        if (g >= a.total) continue;
        const int64_t b = g / a.nR, j = g - b * a.nR;
        const int64_t jm = j % a.Ns;
        out[b * a.n + (j / a.Ns) * a.Ns * a.R + jm + (int64_t)m * a.Ns] = src[c * a.PR + m];
    }
}

__device__ __forceinline__ cdd to_cdd(double re, double im) {
    cdd r;
    r.x = dd_from_double(re);
    r.y = dd_from_double(im);
    return r;
}

__global__ void k_make_twiddles_full(int64_t n, double2* out_d, float2* out_f, cdd* out_x) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s, c;
    sincospi(-2.0 * (double)i / (double)n, &s, &c);
    if (out_d) out_d[i] = make_double2(c, s);
    if (out_f) out_f[i] = make_float2((float)c, (float)s);
    if (out_x) out_x[i] = to_cdd(c, s);
}

// in-place representation changes for the double-float FFTs (16 bytes either way)
__global__ void k_to_dd(double2* buf, int64_t n) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = buf[i];
    reinterpret_cast<cdd*>(buf)[i] = to_cdd(v.x, v.y);
}
__global__ void k_from_dd(double2* buf, int64_t n) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cdd v = reinterpret_cast<const cdd*>(buf)[i];
    buf[i] = make_double2(dd_to_double(v.x), dd_to_double(v.y));
}

__global__ void k_make_twiddles(int64_t n, int64_t B, int64_t nhi, double2* lo_d, double2* hi_d,
                                float2* lo_f, float2* hi_f, cdd* lo_x, cdd* hi_x) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) {
        double s, c;
        sincospi(-2.0 * (double)i / (double)n, &s, &c);
        if (lo_d) lo_d[i] = make_double2(c, s);
        if (lo_f) lo_f[i] = make_float2((float)c, (float)s);
        if (lo_x) lo_x[i] = to_cdd(c, s);
    }
    if (i < nhi) {
        // exponent i*B mod n, exact in integers before the division
        const int64_t e = (i * B) % n;
        double s, c;
        sincospi(-2.0 * (double)e / (double)n, &s, &c);
        if (hi_d) hi_d[i] = make_double2(c, s);
        if (hi_f) hi_f[i] = make_float2((float)c, (float)s);
        if (hi_x) hi_x[i] = to_cdd(c, s);
    }
}

// ---- Bluestein --------------------------------------------------------------
// chirp c_k = e^{+j pi k^2/n}; forward filter h_m = c_m (m in (-n, n)),
// inverse filter conj(h).  Phases are reduced exactly: k^2 mod 2n.
__global__ void k_blue_chirp(int64_t n, int64_t m, double2* chirp_d, float2* chirp_f, cdd* chirp_x, double2* hf,
                             double2* hi) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t k = -1;
    if (i < n) k = i; else if (i > m - n) k = m - i;
    double2 c = make_double2(0.0, 0.0);
    if (k >= 0) {
        const int64_t e = (int64_t)(((unsigned long long)k * (unsigned long long)k) % (unsigned long long)(2 * n));
        double s, co;
        sincospi((double)e / (double)n, &s, &co);
        c = make_double2(co, s);
        if (i < n) {
            if (chirp_d) chirp_d[i] = c;
            if (chirp_f) chirp_f[i] = make_float2((float)co, (float)s);
            if (chirp_x) chirp_x[i] = to_cdd(co, s);
        }
    }
    hf[i] = c;
    hi[i] = make_double2(c.x, -c.y);
}

__global__ void k_scale_c128_to(const double2* in, int64_t m, double s, double2* out_d, float2* out_f, cdd* out_x) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double2 v = in[i];
    v.x *= s; v.y *= s;
    if (out_d) out_d[i] = v;
    if (out_f) out_f[i] = make_float2((float)v.x, (float)v.y);
    if (out_x) out_x[i] = to_cdd(v.x, v.y);
}

template <typename T>
__global__ void k_blue_pre(const c2<T>* __restrict__ x, int64_t n, int64_t m, const c2<T>* __restrict__ chirp,
                           int dir, int64_t batch, c2<T>* __restrict__ a) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * batch) return;
    const int64_t b = i / m, j = i - b * m;
    c2<T> v = mk<T>(0, 0);
    if (j < n) {
        c2<T> c = chirp[j];
        v = dir < 0 ? cmulc(x[b * n + j], c) : cmul(x[b * n + j], c);
    }
    a[i] = v;
}

template <typename T>
__global__ void k_blue_mul(c2<T>* __restrict__ a, const c2<T>* __restrict__ h, int64_t m, int64_t batch) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m * batch) return;
    a[i] = cmul(a[i], h[i % m]);
}

template <typename T>
__global__ void k_blue_post(const c2<T>* __restrict__ a, int64_t n, int64_t m, const c2<T>* __restrict__ chirp,
                            int dir, int64_t batch, c2<T>* __restrict__ x) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * batch) return;
    const int64_t b = i / n, k = i - b * n;
    c2<T> c = chirp[k];
    c2<T> v = a[b * m + k];
    x[i] = dir < 0 ? cmulc(v, c) : cmul(v, c);
}

std::vector<int> factor_small(int64_t n) {
    std::vector<int> f;
    for (int p : {2, 3, 5, 7}) while (n % p == 0) { f.push_back(p); n /= p; }
    return f;
}

// split the prime factors into `k` passes with balanced products (each <= lmax)
bool split_passes(std::vector<int> f, int k, int lmax, std::vector<int64_t>& out) {
    std::sort(f.begin(), f.end(), std::greater<int>());
    out.assign(k, 1);
    for (int p : f) {
        int best = -1;
        for (int i = 0; i < k; ++i)
            if (out[i] * p <= lmax && (best < 0 || out[i] < out[best])) best = i;
        if (best < 0) return false;
        out[best] *= p;
    }
    return true;
}

std::vector<int> sub_radices(int64_t R) {
    std::vector<int> s;
    while (R % 8 == 0) { s.push_back(8); R /= 8; }
    while (R % 4 == 0) { s.push_back(4); R /= 4; }
    while (R % 2 == 0) { s.push_back(2); R /= 2; }
    for (int p : {3, 5, 7}) while (R % p == 0) { s.push_back(p); R /= p; }
    return s;
}

// ---- power-of-two passes ----------------------------------------------------
template <typename T> struct P2Limits;
template <> struct P2Limits<float> { static constexpr int kElems = 4096; static constexpr int kRlogMax = 10; };
template <> struct P2Limits<double> { static constexpr int kElems = 2048; static constexpr int kRlogMax = 8; };
// double-float plans use radix <= 64: their transforms are few (batch 1 to
// eta), so more, lighter threads per pass beat fewer passes
template <> struct P2Limits<dd> { static constexpr int kElems = 2048; static constexpr int kRlogMax = 6; };

inline int r1_log_of(int rlog) { return (rlog + 1) / 2; }   // R1 >= R2, R1 <= 2 R2

template <typename T>
int p2_C_log(int rlog) {
    const int r2log = rlog - r1_log_of(rlog);
    int c = P2Limits<T>::kElems >> rlog;
    c = std::min(c, 256 >> r2log);
    int cl = 0;
    while ((1 << (cl + 1)) <= c) ++cl;
    return cl;
}

// split n = 2^L into passes of radix 2^r (r <= kRlogMax), balanced; every
// pass of a multi-pass plan must own whole columns (C <= n/R)
template <typename T>
bool plan_p2(int L, std::vector<int>& rl) {
    if (L < 1) return false;
    const int rmax = P2Limits<T>::kRlogMax;
    const int k = (L + rmax - 1) / rmax;
    rl.assign(k, L / k);
    for (int i = 0; i < L % k; ++i) rl[i] += 1;
    if (k > 1)
        for (int r : rl)
            if (p2_C_log<T>(r) > L - r) return false;
    return true;
}

template <typename T>
nufft_status launch_p2(int rlog, const c2<T>* in, c2<T>* out, p2::Args a, const c2<T>* lo, const c2<T>* hi, int dir,
                       cudaStream_t s) {
    const int r1 = 1 << r1_log_of(rlog), r2 = 1 << (rlog - r1_log_of(rlog));
    const int C = 1 << a.C_log;
    const int PR = r1 * (r2 + 1) + 1;
    const size_t smem = (size_t)C * PR * sizeof(c2<T>);
    const unsigned blocks = (unsigned)((a.total + C - 1) / C);
    const unsigned threads = (unsigned)(C * r2);
#define P2_CASE(RL, A, B)                                                                                   \
    case RL: {                                                                                              \
        auto kern = p2::k_fft_p2<T, A, B>;                                                                  \
        NUFFT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        launch_k(kern, blocks, threads, smem, s, in, out, a, lo, hi, dir);                                        \
        break;                                                                                              \
    }
    switch (rlog) {
        P2_CASE(1, 2, 1)
        P2_CASE(2, 2, 2)
        P2_CASE(3, 4, 2)
        P2_CASE(4, 4, 4)
        P2_CASE(5, 8, 4)
        P2_CASE(6, 8, 8)
        P2_CASE(7, 16, 8)
        P2_CASE(8, 16, 16)
        default:
            if constexpr (sizeof(T) == 4) {
                switch (rlog) {
                    P2_CASE(9, 32, 16)
                    P2_CASE(10, 32, 32)
                    default: return fail(NUFFT_ERR_ARG, "no power-of-two pass for radix 2^%d", rlog);
                }
            } else {
                return fail(NUFFT_ERR_ARG, "no power-of-two pass for radix 2^%d", rlog);
            }
    }
#undef P2_CASE
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

template <typename T, int A, int B>
nufft_status launch_p2s_one(const c2<T>* in, c2<T>* out, p2::SArgs a, const c2<T>* tw, int dir, cudaStream_t s) {
    using G = p2::SCfg<T, A, B>;
    auto kern = p2::k_fft_p2s<T, A, B>;
    const size_t smem = 2 * (size_t)G::R * G::C * sizeof(c2<T>);
    static int per_sm = 0;   // resident CTAs per SM for this instantiation (device-independent enough)
    if (!per_sm) {
        NUFFT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int b = 0;
        NUFFT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, G::TH, smem));
        per_sm = std::max(1, b);
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(a.ntiles, per_sm * std::max(1, sms));
    launch_k(kern, grid, G::TH, smem, s, in, out, a, tw, dir);
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

template <typename T>
nufft_status launch_p2s(int rlog, const c2<T>* in, c2<T>* out, p2::SArgs a, const c2<T>* tw, int dir,
                        cudaStream_t s) {
    switch (rlog) {
        case 4: return launch_p2s_one<T, 4, 4>(in, out, a, tw, dir, s);
        case 5: return launch_p2s_one<T, 8, 4>(in, out, a, tw, dir, s);
        case 6: return launch_p2s_one<T, 8, 8>(in, out, a, tw, dir, s);
        case 7: return launch_p2s_one<T, 16, 8>(in, out, a, tw, dir, s);
        case 8: return launch_p2s_one<T, 16, 16>(in, out, a, tw, dir, s);
        default:
            if constexpr (sizeof(T) == 4) {
                if (rlog == 9) return launch_p2s_one<T, 32, 16>(in, out, a, tw, dir, s);
                if (rlog == 10) return launch_p2s_one<T, 32, 32>(in, out, a, tw, dir, s);
            }
            return fail(NUFFT_ERR_ARG, "no streaming pass for radix 2^%d", rlog);
    }
}

// ---- TMA-fed float32 passes ------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// the tile counter set of the next TMA-fed pass on device `dev`: one sequence
// per device (the counters live in each device's memory, and a launch zeroes
// the set it will reuse on its own device) shared by every instantiation of
// the pass, so consecutive launches never share a set
static int p2t_next_slot(int dev) {
    static std::atomic<unsigned> next[128];
    return (int)(next[(unsigned)dev & 127u].fetch_add(1u, std::memory_order_relaxed) % (unsigned)p2t::kTileSlots);
}

template <int R1, int R2, bool FUSE = false>
nufft_status launch_p2t_one(const float2* in, float2* out, const p2t::TArgs& ta, int64_t batch, const float2* tw,
                            int dir, cudaStream_t s) {
    using G = p2t::TCfg<R1, R2>;
    // the pass's inputs as a 4-D array (j, k2, k1, vector): x[v n + j + (k1 R2 + k2) n/R]
    const uint64_t nR = 1ull << (ta.n_log - ta.R_log);
    CUtensorMap tm;
    cuuint64_t dims[4] = {nR, (cuuint64_t)R2, (cuuint64_t)R1, (cuuint64_t)batch};
    cuuint64_t strides[3] = {nR * sizeof(float2), (cuuint64_t)R2 * nR * sizeof(float2),
                             (1ull << ta.n_log) * sizeof(float2)};
    cuuint32_t box[4] = {(cuuint32_t)G::C, (cuuint32_t)R2, (cuuint32_t)(ta.lop == 3 ? R1 / 4 : R1), 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    if (tma_encoder()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, const_cast<float2*>(in), dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(NUFFT_ERR_CUDA, "tensor map for a %d x %d FFT pass rejected", R1, R2);
    auto kern = p2t::k_fft_p2t<R1, R2, FUSE>;
    constexpr size_t smem = p2t::smem_bytes<R1, R2>();
    static int per_sm = 0;
    if (!per_sm) {
        NUFFT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int b = 0;
        NUFFT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, G::TH, smem));
        per_sm = std::max(1, b);
    }
    int dev = 0, sms = 0;
    NUFFT_CUDA_TRY(cudaGetDevice(&dev));
    NUFFT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(ta.ntiles, per_sm * std::max(1, sms));
    p2t::TArgs tl = ta;
    tl.slot = p2t_next_slot(dev);
    launch_k(kern, grid, G::TH, smem, s, tm, out, tl, tw, dir);
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

// Run one float32 pass on the TMA-fed kernel when it applies (radix 256 or
// 512 in a multi-pass plan, whole tiles inside a vector, no gather on the
// loads); *done tells whether it ran.
template <typename T>
nufft_status try_p2t(const FFTPlan& p, const c2<T>* in, c2<T>* out, const p2::Args& a, int64_t batch, int dir,
                     cudaStream_t s, bool* done) {
    *done = false;
    if constexpr (sizeof(T) != 4) {
        return NUFFT_OK;
    } else {
        if (!p.tw_full || p.p2_rlog.size() < 2 || (a.R_log != 8 && a.R_log != 9)) return NUFFT_OK;
        if (a.lop != 0 && a.lop != 2 && a.lop != 3) return NUFFT_OK;
        if (a.lop == 3 && a.Ns_log != 0) return NUFFT_OK;
        if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15)) return NUFFT_OK;
        const int clog = p2_C_log<float>(a.R_log);
        if (clog > a.n_log - a.R_log) return NUFFT_OK;                       // a tile stays inside one vector
        if (a.Ns_log != 0 && a.Ns_log < clog) return NUFFT_OK;                // stores: direct or one contiguous block
        if (a.Ns_log < clog && a.sop != 0) return NUFFT_OK;
        if (batch > (1ll << 31) / ((1ll << (a.n_log - a.R_log)) >> clog)) return NUFFT_OK;
        if (!tma_encoder()) return NUFFT_OK;
        p2t::TArgs ta;
        ta.n_log = a.n_log;
        ta.R_log = a.R_log;
        ta.Ns_log = a.Ns_log;
        ta.C_log = clog;
        ta.ntiles = (int)((batch << (a.n_log - a.R_log)) >> clog);
        ta.lop = a.lop;
        ta.sop = a.sop;
        ta.fac_in = static_cast<const float*>(a.fac_in);
        ta.mulc = static_cast<const float2*>(a.mulc);
        ta.fac_out = static_cast<const float*>(a.fac_out);
        ta.out_bs = a.out_bs;
        ta.off = a.sel_off;
        ta.len = a.sel_len;
        ta.fmul = nullptr;
        const float2* tw = static_cast<const float2*>(p.tw_full);
        nufft_status st = (a.R_log == 8) ? launch_p2t_one<16, 16>(in, out, ta, batch, tw, dir, s)
                                         : launch_p2t_one<32, 16>(in, out, ta, batch, tw, dir, s);
        *done = (st == NUFFT_OK);
        return st;
    }
}

// every pass of the plan runs on the streaming kernel (8-byte scalars)
template <typename T>
bool p2s_all(const FFTPlan& p) {
    if (sizeof(T) != 8 || !p.tw_full || p.p2_rlog.size() < 2) return false;
    int L = 0;
    while (((int64_t)1 << L) < p.n) ++L;
    for (int rl : p.p2_rlog)
        if (rl < 4 || p2_C_log<T>(rl) > L - rl) return false;
    return true;
}

template <typename T>
nufft_status exec_p2(const FFTPlan& p, c2<T>* buf, c2<T>* work, int64_t batch, int dir, cudaStream_t s,
                     c2<T>** result, int cvt_in = 0, int cvt_out = 0) {
    const c2<T>* lo = static_cast<const c2<T>*>(p.tw_lo);
    const c2<T>* hi = static_cast<const c2<T>*>(p.tw_hi);
    int L = 0;
    while (((int64_t)1 << L) < p.n) ++L;
    c2<T>* src = buf;
    c2<T>* dst = (p.p2_rlog.size() == 1) ? buf : work;
    int ns_log = 0;
    for (size_t i = 0; i < p.p2_rlog.size(); ++i) {
        const int rl = p.p2_rlog[i];
        p2::Args a;
        a.n_log = L;
        a.R_log = rl;
        a.Ns_log = ns_log;
        a.C_log = p2_C_log<T>(rl);
        a.total = (int)(batch << (L - rl));
        a.shift = p.shift;
        a.tw_full = p.tw_full;
        a.lop = a.sop = 0;
        a.src = a.fac_in = a.mulc = a.fac_out = nullptr;
        a.src_bs = a.ns = a.K0 = 0;
        a.out_bs = a.sel_off = a.sel_len = 0;
        {
            Launch Lk(s, K_FFT, 2.0 * (double)p.n * (double)batch * sizeof(c2<T>), sizeof(T) == 8);
            const int clog = p2_C_log<T>(rl);
            // float32 radix-256/512 passes of multi-pass plans: TMA-fed tiles;
            // float64 passes stream tiles through shared memory with cp.async
            // (their float64 arithmetic is the limit; prefetching the next tile
            // hides the loads); other float32 passes load straight into
            // registers from many resident CTAs
            bool done = false;
            nufft_status st = try_p2t<T>(p, src, dst, a, batch, dir, s, &done);
            if (st == NUFFT_OK && !done) {
                if (sizeof(T) == 8 && p.tw_full && p.p2_rlog.size() > 1 && rl >= 4 && clog <= L - rl) {
                    p2::SArgs sa;
                    sa.n_log = L;
                    sa.R_log = rl;
                    sa.Ns_log = ns_log;
                    sa.ntiles = (int)((batch << (L - rl)) >> clog);
                    sa.cvt_in = (i == 0) ? cvt_in : 0;
                    sa.cvt_out = (i + 1 == p.p2_rlog.size()) ? cvt_out : 0;
                    st = launch_p2s<T>(rl, src, dst, sa, static_cast<const c2<T>*>(p.tw_full), dir, s);
                } else {
                    st = launch_p2<T>(rl, src, dst, a, lo, hi, dir, s);
                }
            }
            if (st != NUFFT_OK) return st;
        }
        ns_log += rl;
        src = dst;
        dst = (dst == buf) ? work : buf;
    }
    *result = src;
    return NUFFT_OK;
}

template <typename T>
nufft_status make_passes(FFTPlan& p) {
    const int64_t n = p.n;
    if (n >= 2 && (n & (n - 1)) == 0 && n <= ((int64_t)1 << 30)) {
        int L = 0;
        while (((int64_t)1 << L) < n) ++L;
        if (plan_p2<T>(L, p.p2_rlog)) return NUFFT_OK;
        p.p2_rlog.clear();
    }
    std::vector<int> f = factor_small(n);
    std::vector<int64_t> radices;
    if (n <= FftLimits<T>::kElems) {
        radices.push_back(n);
    } else {
        int k = 2;
        while (!split_passes(f, k, FftLimits<T>::kLmax, radices)) ++k;
    }
    int64_t Ns = 1;
    for (int64_t R : radices) {
        FFTPass ps;
        ps.R = (int)R;
        ps.Ns = Ns;
        std::vector<int> sr = sub_radices(R);
        ps.nsub = (int)sr.size();
        for (int i = 0; i < ps.nsub; ++i) ps.sub[i] = sr[i];
        if (radices.size() == 1) ps.C = std::max<int64_t>(1, FftLimits<T>::kElems / R);
        else ps.C = 16;
        p.passes.push_back(ps);
        Ns *= R;
    }
    return NUFFT_OK;
}

template <typename T>
nufft_status exec_passes(const FFTPlan& p, c2<T>* buf, c2<T>* work, int64_t batch, int dir, cudaStream_t s,
                         c2<T>** result) {
    const c2<T>* lo = static_cast<const c2<T>*>(p.tw_lo);
    const c2<T>* hi = static_cast<const c2<T>*>(p.tw_hi);
    c2<T>* src = buf;
    c2<T>* dst = (p.passes.size() == 1) ? buf : work;
    for (size_t i = 0; i < p.passes.size(); ++i) {
        const FFTPass& ps = p.passes[i];
        PassArgs a;
        a.n = p.n; a.R = ps.R; a.nR = p.n / ps.R; a.Ns = ps.Ns;
        a.total = batch * a.nR;
        a.C = (int)std::min<int64_t>(ps.C, a.total);
        a.PR = ps.R + 1;
        a.nsub = ps.nsub;
        for (int q = 0; q < 12; ++q) a.sub[q] = ps.sub[q];
        a.in_cfast = (a.nR >= a.C) ? 1 : 0;
        a.out_cfast = (ps.Ns >= a.C) ? 1 : 0;
        a.shift = p.shift;
        a.mask = ((int64_t)1 << p.shift) - 1;
        const size_t smem = 2 * (size_t)a.C * a.PR * sizeof(c2<T>);
        const int64_t blocks = (a.total + a.C - 1) / a.C;
        NUFFT_CUDA_TRY(cudaFuncSetAttribute(k_fft_pass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        {
            Launch L(s, K_FFT, 2.0 * (double)p.n * (double)batch * sizeof(c2<T>), sizeof(T) == 8);
            launch_k(k_fft_pass<T>, (unsigned)blocks, kThreads, smem, s, src, dst, a, lo, hi, dir);
        }
        NUFFT_CUDA_TRY(cudaGetLastError());
        src = dst;
        dst = (dst == buf) ? work : buf;
    }
    *result = src;
    return NUFFT_OK;
}

template <typename T>
nufft_status exec_p2_hooked(const FFTPlan& p, const c2<T>* in, c2<T>* work, c2<T>* out, int64_t batch, int dir,
                            const FFTHooks& h, cudaStream_t s) {
    const c2<T>* lo = static_cast<const c2<T>*>(p.tw_lo);
    const c2<T>* hi = static_cast<const c2<T>*>(p.tw_hi);
    int L = 0;
    while (((int64_t)1 << L) < p.n) ++L;
    const int k = (int)p.p2_rlog.size();
    const c2<T>* src = in;
    int ns_log = 0;
    for (int i = 0; i < k; ++i) {
        const int rl = p.p2_rlog[i];
        c2<T>* dst = ((k - 1 - i) % 2 == 0) ? out : work;
        p2::Args a;
        a.n_log = L;
        a.R_log = rl;
        a.Ns_log = ns_log;
        a.C_log = p2_C_log<T>(rl);
        a.total = (int)(batch << (L - rl));
        a.shift = p.shift;
        a.tw_full = p.tw_full;
        a.lop = (i == 0) ? h.lop : 0;
        a.sop = (i == k - 1) ? h.sop : 0;
        a.src = h.src;
        a.src_bs = h.src_bs;
        a.ns = h.ns;
        a.K0 = h.K0;
        a.fac_in = h.fac_in;
        a.mulc = h.mulc;
        a.fac_out = h.fac_out;
        a.out_bs = h.out_bs;
        a.sel_off = a.sel_len = 0;
        if (a.sop == 3) { a.sel_off = h.K0; a.sel_len = h.P; }
        if (a.sop == 4) { a.sel_off = h.K0; a.sel_len = h.ns; }
        {
            // algorithmic bytes: one read and one write of the vectors (the
            // selecting store writes P of the n outputs, the half-support
            // load reads n/2 of the n inputs)
            const double wr = (a.sop == 3) ? (double)h.P : (double)p.n;
            const double rd = (a.lop == 3) ? 0.5 * (double)p.n : (double)p.n;
            Launch Lk(s, K_FFT, (rd + wr) * (double)batch * sizeof(c2<T>), sizeof(T) == 8);
            bool done = false;
            nufft_status st = try_p2t<T>(p, src, dst, a, batch, dir, s, &done);
            if (st == NUFFT_OK && !done) {
                if (a.sop >= 3 || a.lop == 3)
                    return fail(NUFFT_ERR_ARG, "scattering FFT stores and half-support loads need the TMA-fed pass");
                st = launch_p2<T>(rl, src, dst, a, lo, hi, dir, s);
            }
            if (st != NUFFT_OK) return st;
        }
        ns_log += rl;
        src = dst;
    }
    return NUFFT_OK;
}

}  // namespace

template <typename T>
bool fft_scatter_supported(const FFTPlan& p) {
    if constexpr (sizeof(T) != 4) {
        return false;
    } else {
        if (p.p2_rlog.size() != 2 || !p.tw_full || !tma_encoder()) return false;
        int L = 0;
        while (((int64_t)1 << L) < p.n) ++L;
        int ns_log = 0;
        for (int rl : p.p2_rlog) {
            if (rl != 8 && rl != 9) return false;
            const int clog = p2_C_log<float>(rl);
            if (clog > L - rl || (ns_log != 0 && ns_log < clog)) return false;
            ns_log += rl;
        }
        return true;
    }
}
template bool fft_scatter_supported<float>(const FFTPlan&);
template bool fft_scatter_supported<double>(const FFTPlan&);

template <typename T>
bool fft_conv_supported(const FFTPlan& p) {
    return sizeof(T) == 4 && p.p2_rlog.size() == 2 && p.p2_rlog[0] == 8 && p.p2_rlog[1] == 8 &&
           fft_scatter_supported<T>(p);
}
template bool fft_conv_supported<float>(const FFTPlan&);
template bool fft_conv_supported<double>(const FFTPlan&);

template <typename T>
nufft_status fft_exec_conv(const FFTPlan& p, const c2<T>* in, c2<T>* w1, c2<T>* w2, c2<T>* out, int64_t batch,
                           int dir, const c2<T>* fmul, const FFTHooks& h, cudaStream_t s) {
    if constexpr (sizeof(T) != 4) {
        return fail(NUFFT_ERR_ARG, "the fused transform pair is float32 only");
    } else {
        if (!fft_conv_supported<T>(p)) return fail(NUFFT_ERR_ARG, "the fused transform pair needs n = 256 x 256");
        if (batch <= 0) return NUFFT_OK;
        const int L = 16;
        const double vec = (double)p.n * (double)batch * sizeof(c2<T>);
        // first transform, pass 1 (loads hook h.lop)
        FFTHooks h1;
        h1.lop = h.lop; h1.fac_in = h.fac_in;
        {
            p2::Args a{};
            a.n_log = L; a.R_log = 8; a.Ns_log = 0; a.C_log = p2_C_log<T>(8);
            a.total = (int)(batch << 8); a.shift = p.shift; a.tw_full = p.tw_full;
            a.lop = h.lop; a.sop = 0; a.fac_in = h.fac_in;
            Launch Lk(s, K_FFT, 2.0 * vec);
            bool done = false;
            nufft_status st = try_p2t<T>(p, in, w1, a, batch, dir, s, &done);
            if (st != NUFFT_OK) return st;
            if (!done) return fail(NUFFT_ERR_ARG, "fused transform pair: TMA pass unavailable");
        }
        // first transform's pass 2, x fmul, second transform's pass 1
        {
            Launch Lk(s, K_FFT, 2.0 * vec);
            p2t::TArgs ta{};
            ta.n_log = L; ta.R_log = 8; ta.Ns_log = 8; ta.C_log = p2_C_log<float>(8);
            ta.ntiles = (int)((batch << 8) >> ta.C_log);
            ta.fmul = reinterpret_cast<const float2*>(fmul);
            nufft_status st = launch_p2t_one<16, 16, true>(reinterpret_cast<const float2*>(w1),
                                                           reinterpret_cast<float2*>(w2), ta, batch,
                                                           static_cast<const float2*>(p.tw_full), dir, s);
            if (st != NUFFT_OK) return st;
        }
        // second transform, pass 2 (stores hook h.sop)
        {
            p2::Args a{};
            a.n_log = L; a.R_log = 8; a.Ns_log = 8; a.C_log = p2_C_log<T>(8);
            a.total = (int)(batch << 8); a.shift = p.shift; a.tw_full = p.tw_full;
            a.lop = 0; a.sop = h.sop; a.mulc = h.mulc; a.fac_out = h.fac_out; a.out_bs = h.out_bs;
            if (a.sop == 3) { a.sel_off = h.K0; a.sel_len = h.P; }
            if (a.sop == 4) { a.sel_off = h.K0; a.sel_len = h.ns; }
            Launch Lk(s, K_FFT, 2.0 * vec);
            bool done = false;
            nufft_status st = try_p2t<T>(p, w2, out, a, batch, -dir, s, &done);
            if (st != NUFFT_OK) return st;
            if (!done) return fail(NUFFT_ERR_ARG, "fused transform pair: TMA pass unavailable");
        }
        return NUFFT_OK;
    }
}
template nufft_status fft_exec_conv<float>(const FFTPlan&, const float2*, float2*, float2*, float2*, int64_t, int,
                                           const float2*, const FFTHooks&, cudaStream_t);
template nufft_status fft_exec_conv<double>(const FFTPlan&, const double2*, double2*, double2*, double2*, int64_t,
                                            int, const double2*, const FFTHooks&, cudaStream_t);

template <typename T>
bool fft_hooks_supported(const FFTPlan& p) {
    if (p.p2_rlog.size() < 2) return false;
    int L = 0;
    while (((int64_t)1 << L) < p.n) ++L;
    for (int rl : p.p2_rlog)
        if (p2_C_log<T>(rl) > L - rl) return false;
    return true;
}

template <typename T>
nufft_status fft_exec_hooked(const FFTPlan& p, const c2<T>* in, c2<T>* work, c2<T>* out, int64_t batch, int dir,
                             const FFTHooks& h, cudaStream_t s) {
    if (!fft_hooks_supported<T>(p)) return fail(NUFFT_ERR_ARG, "fused FFT stages need a multi-pass power-of-two plan");
    if (batch <= 0) return NUFFT_OK;
    return exec_p2_hooked<T>(p, in, work, out, batch, dir, h, s);
}

template bool fft_hooks_supported<float>(const FFTPlan&);
template bool fft_hooks_supported<double>(const FFTPlan&);
template nufft_status fft_exec_hooked<float>(const FFTPlan&, const float2*, float2*, float2*, int64_t, int,
                                             const FFTHooks&, cudaStream_t);
template nufft_status fft_exec_hooked<double>(const FFTPlan&, const double2*, double2*, double2*, int64_t, int,
                                              const FFTHooks&, cudaStream_t);

bool is_smooth(int64_t n) {
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7}) while (n % p == 0) n /= p;
    return n == 1;
}

int64_t next_smooth(int64_t n) {
    if (n < 1) n = 1;
    while (!is_smooth(n)) ++n;
    return n;
}

FFTPlan::~FFTPlan() {
    cudaFree(tw_full);
    cudaFree(tw_lo);
    cudaFree(tw_hi);
    cudaFree(chirp);
    cudaFree(chirp_hat_fwd);
    cudaFree(chirp_hat_inv);
}

int64_t fft_work_elems(const FFTPlan& p) { return p.bluestein ? 2 * p.m : p.n; }

namespace {
// a wait on a barrier phase that nothing completes: the bounded wait of the
// pass kernels gives up and counts the expiry (test hook)
__global__ void k_debug_wait_expiry() {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        p2t::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!p2t::mbar_wait(&bar, 0)) atomicAdd(&g_wait_expired, 1);
    }
}
}  // namespace

nufft_status fft_wait_status(cudaStream_t s) {
    int expired = 0;
    NUFFT_CUDA_TRY(cudaMemcpyFromSymbolAsync(&expired, g_wait_expired, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    if (expired == 0) return NUFFT_OK;
    const int zero = 0;
    NUFFT_CUDA_TRY(cudaMemcpyToSymbolAsync(g_wait_expired, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return fail(NUFFT_ERR_TIMEOUT, "%d FFT pass tile wait(s) expired", expired);
}

// passes of the shared-memory double-float kernel: n = 2^L, L >= 11, split into
// balanced radices 2^5 .. 2^10 (at least two passes, so that every pass has
// n/R >= 2 columns)
// batches up to this many points take the shared-memory radix-4 kernel (for
// few vectors its threads are what the pass needs; for the all-float64 path's
// batches its radix-1024 passes save a pass over the radix-64 streaming
// ones); beyond it the streaming passes
constexpr int64_t kDdqMaxElems = (int64_t)1 << 26;

static void plan_ddq(int64_t n, std::vector<int>& rl) {
    rl.clear();
    int L = 0;
    while (((int64_t)1 << L) < n) ++L;
    if (L < 11 || ((int64_t)1 << L) != n) return;
    const int k = (L + 9) / 10;
    rl.assign(k, L / k);
    for (int i = 0; i < L % k; ++i) rl[i] += 1;
}

static nufft_status exec_ddq(const FFTPlan& p, cdd* buf, cdd* work, int64_t batch, int dir, cudaStream_t s, cdd** result,
                             int cvt_in, int cvt_out) {
    int L = 0;
    while (((int64_t)1 << L) < p.n) ++L;
    const cdd* tw = static_cast<const cdd*>(p.tw_full);
    cdd* src = buf;
    cdd* dst = work;
    int ns_log = 0;
    const size_t k = p.q_rlog.size();
    for (size_t i = 0; i < k; ++i) {
        const int rl = p.q_rlog[i];
        ddq::QArgs a;
        a.n_log = L;
        a.Ns_log = ns_log;
        a.cvt_in = (i == 0) ? cvt_in : 0;
        a.cvt_out = (i + 1 == k) ? cvt_out : 0;
        const int64_t grid = (batch << (L - rl)) / ddq::kCols;
        const unsigned th = (unsigned)(ddq::kCols * (1 << rl) / 4);
        {
            Launch Lk(s, K_FFT, 2.0 * (double)p.n * (double)batch * sizeof(cdd), true);
            switch (rl) {
                case 5: launch_k(ddq::k_fft_ddq<5>, (unsigned)grid, th, 0, s, src, dst, a, tw, dir); break;
                case 6: launch_k(ddq::k_fft_ddq<6>, (unsigned)grid, th, 0, s, src, dst, a, tw, dir); break;
                case 7: launch_k(ddq::k_fft_ddq<7>, (unsigned)grid, th, 0, s, src, dst, a, tw, dir); break;
                case 8: launch_k(ddq::k_fft_ddq<8>, (unsigned)grid, th, 0, s, src, dst, a, tw, dir); break;
                case 9: launch_k(ddq::k_fft_ddq<9>, (unsigned)grid, th, 0, s, src, dst, a, tw, dir); break;
                case 10: launch_k(ddq::k_fft_ddq<10>, (unsigned)grid, th, 0, s, src, dst, a, tw, dir); break;
                default: return fail(NUFFT_ERR_ARG, "no few-vector pass for radix 2^%d", rl);
            }
        }
        NUFFT_CUDA_TRY(cudaGetLastError());
        ns_log += rl;
        src = dst;
        dst = (dst == buf) ? work : buf;
    }
    *result = src;
    return NUFFT_OK;
}

nufft_status fft_make(FFTPlan& p, int64_t n, int prec, cudaStream_t s) {
    p.n = n;
    p.prec = prec;
    if (n < 1) return fail(NUFFT_ERR_ARG, "FFT length %lld < 1", (long long)n);
    if (!is_smooth(n)) {
        p.bluestein = true;
        p.m = next_smooth(2 * n - 1);
        p.sub.reset(new FFTPlan());
        nufft_status st = fft_make(*p.sub, p.m, prec, s);
        if (st != NUFFT_OK) return st;
        const int64_t m = p.m;
        double2 *hf = nullptr, *hi = nullptr, *work = nullptr;
        NUFFT_CUDA_TRY(cudaMalloc(&hf, sizeof(double2) * m));
        NUFFT_CUDA_TRY(cudaMalloc(&hi, sizeof(double2) * m));
        NUFFT_CUDA_TRY(cudaMalloc(&work, sizeof(double2) * fft_work_elems(*p.sub)));
        const size_t es = prec >= 2 ? sizeof(double2) : sizeof(float2);
        NUFFT_CUDA_TRY(cudaMalloc(&p.chirp, es * n));
        NUFFT_CUDA_TRY(cudaMalloc(&p.chirp_hat_fwd, es * m));
        NUFFT_CUDA_TRY(cudaMalloc(&p.chirp_hat_inv, es * m));
        const int tb = 256;
        Launch Lc(s, K_PLAN_TABLE, 48.0 * m);
        launch_k(k_blue_chirp, (unsigned)((m + tb - 1) / tb), tb, 0, s, 
            n, m, prec == 2 ? (double2*)p.chirp : nullptr, prec == 1 ? (float2*)p.chirp : nullptr,
            prec == 3 ? (cdd*)p.chirp : nullptr, hf, hi);
        NUFFT_CUDA_TRY(cudaGetLastError());
        // the filter spectra are always formed in float64
        FFTPlan p64;
        st = fft_make(p64, m, 2, s);
        if (st != NUFFT_OK) return st;
        double2* res = nullptr;
        for (int which = 0; which < 2; ++which) {
            double2* h = which == 0 ? hf : hi;
            st = fft_exec<double>(p64, h, work, 1, -1, s, &res);
            if (st != NUFFT_OK) return st;
            void* dst = which == 0 ? p.chirp_hat_fwd : p.chirp_hat_inv;
            Launch Ls(s, K_PLAN_TABLE, 32.0 * m);
            launch_k(k_scale_c128_to, (unsigned)((m + tb - 1) / tb), tb, 0, s, 
                res, m, 1.0 / (double)m, prec == 2 ? (double2*)dst : nullptr, prec == 1 ? (float2*)dst : nullptr,
                prec == 3 ? (cdd*)dst : nullptr);
            NUFFT_CUDA_TRY(cudaGetLastError());
        }
        NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(hf);
        cudaFree(hi);
        cudaFree(work);
        return NUFFT_OK;
    }
    // two-level twiddle table
    int shift = 0;
    while (((int64_t)1 << (2 * shift)) < n) ++shift;
    p.shift = shift;
    const int64_t B = (int64_t)1 << shift;
    const int64_t nhi = (n + B - 1) / B;
    const size_t es = prec >= 2 ? sizeof(double2) : sizeof(float2);
    NUFFT_CUDA_TRY(cudaMalloc(&p.tw_lo, es * B));
    NUFFT_CUDA_TRY(cudaMalloc(&p.tw_hi, es * nhi));
    const int64_t cnt = std::max(B, nhi);
    Launch Lt(s, K_PLAN_TABLE, 16.0 * (B + nhi));
    launch_k(k_make_twiddles, (unsigned)((cnt + 255) / 256), 256, 0, s, 
        n, B, nhi, prec == 2 ? (double2*)p.tw_lo : nullptr, prec == 2 ? (double2*)p.tw_hi : nullptr,
        prec == 1 ? (float2*)p.tw_lo : nullptr, prec == 1 ? (float2*)p.tw_hi : nullptr,
        prec == 3 ? (cdd*)p.tw_lo : nullptr, prec == 3 ? (cdd*)p.tw_hi : nullptr);
    NUFFT_CUDA_TRY(cudaGetLastError());
    if (n >= 2 && (n & (n - 1)) == 0 && n <= ((int64_t)1 << 24)) {
        NUFFT_CUDA_TRY(cudaMalloc(&p.tw_full, es * n));
        Launch Lf(s, K_PLAN_TABLE, 16.0 * n);
        launch_k(k_make_twiddles_full, (unsigned)((n + 255) / 256), 256, 0, s, 
            n, prec == 2 ? (double2*)p.tw_full : nullptr, prec == 1 ? (float2*)p.tw_full : nullptr,
            prec == 3 ? (cdd*)p.tw_full : nullptr);
        NUFFT_CUDA_TRY(cudaGetLastError());
    }
    nufft_status st = prec == 1 ? make_passes<float>(p) : prec == 2 ? make_passes<double>(p) : make_passes<dd>(p);
    if (st == NUFFT_OK && prec == 3 && p.tw_full) plan_ddq(n, p.q_rlog);
    return st;
}

template <typename T>
nufft_status fft_exec(const FFTPlan& p, c2<T>* buf, c2<T>* work, int64_t batch, int dir, cudaStream_t s,
                      c2<T>** result) {
    if (batch <= 0) { *result = buf; return NUFFT_OK; }
    if (!p.p2_rlog.empty()) return exec_p2<T>(p, buf, work, batch, dir, s, result);
    if (!p.bluestein) return exec_passes<T>(p, buf, work, batch, dir, s, result);
    const int64_t n = p.n, m = p.m;
    c2<T>* a = work;
    c2<T>* aw = work + m * batch;
    const c2<T>* chirp = static_cast<const c2<T>*>(p.chirp);
    const int tb = 256;
    { Launch L(s, K_BLUESTEIN, (double)batch * (n + m) * sizeof(c2<T>) + n * sizeof(c2<T>), sizeof(T) == 8);
    launch_k(k_blue_pre<T>, (unsigned)((m * batch + tb - 1) / tb), tb, 0, s, buf, n, m, chirp, dir, batch, a); }
    NUFFT_CUDA_TRY(cudaGetLastError());
    c2<T>* r = nullptr;
    nufft_status st = p.sub->p2_rlog.empty() ? exec_passes<T>(*p.sub, a, aw, batch, -1, s, &r)
                                                : exec_p2<T>(*p.sub, a, aw, batch, -1, s, &r);
    if (st != NUFFT_OK) return st;
    const c2<T>* h = static_cast<const c2<T>*>(dir < 0 ? p.chirp_hat_fwd : p.chirp_hat_inv);
    { Launch L(s, K_BLUESTEIN, (2.0 * batch + 1.0) * m * sizeof(c2<T>), sizeof(T) == 8);
      launch_k(k_blue_mul<T>, (unsigned)((m * batch + tb - 1) / tb), tb, 0, s, r, h, m, batch); }
    NUFFT_CUDA_TRY(cudaGetLastError());
    c2<T>* r2 = nullptr;
    st = p.sub->p2_rlog.empty() ? exec_passes<T>(*p.sub, r, r == a ? aw : a, batch, +1, s, &r2)
                                : exec_p2<T>(*p.sub, r, r == a ? aw : a, batch, +1, s, &r2);
    if (st != NUFFT_OK) return st;
    { Launch L(s, K_BLUESTEIN, (2.0 * batch + 1.0) * n * sizeof(c2<T>), sizeof(T) == 8);
      launch_k(k_blue_post<T>, (unsigned)((n * batch + tb - 1) / tb), tb, 0, s, r2, n, m, chirp, dir, batch, buf); }
    NUFFT_CUDA_TRY(cudaGetLastError());
    *result = buf;
    return NUFFT_OK;
}

template nufft_status fft_exec<float>(const FFTPlan&, float2*, float2*, int64_t, int, cudaStream_t, float2**);
template nufft_status fft_exec<dd>(const FFTPlan&, cdd*, cdd*, int64_t, int, cudaStream_t, cdd**);

// float64 data through a double-float plan: convert in place, transform,
// convert the result back in place
nufft_status fft_exec_dd(const FFTPlan& p, double2* buf, double2* work, int64_t batch, int dir, cudaStream_t s,
                         double2** result, int io) {
    const int cvt_in = (io & kDdIn) ? 0 : 1, cvt_out = (io & kDdOut) ? 0 : 1;
    if (batch > 0 && !p.q_rlog.empty() && batch * p.n <= kDdqMaxElems) {
        // the shared-memory radix-4 passes, converting on the first pass's
        // loads and the last pass's stores
        cdd* r = nullptr;
        nufft_status st = exec_ddq(p, reinterpret_cast<cdd*>(buf), reinterpret_cast<cdd*>(work), batch, dir, s, &r,
                                   cvt_in, cvt_out);
        if (st != NUFFT_OK) return st;
        *result = reinterpret_cast<double2*>(r);
        return NUFFT_OK;
    }
    if (batch > 0 && p2s_all<dd>(p)) {
        // the first pass converts on its loads, the last on its stores
        cdd* r = nullptr;
        nufft_status st = exec_p2<dd>(p, reinterpret_cast<cdd*>(buf), reinterpret_cast<cdd*>(work), batch, dir, s, &r,
                                      cvt_in, cvt_out);
        if (st != NUFFT_OK) return st;
        *result = reinterpret_cast<double2*>(r);
        return NUFFT_OK;
    }
    const int64_t cnt = p.n * batch;
    const unsigned nb = (unsigned)((cnt + 255) / 256);
    if (cvt_in) {
        Launch L(s, K_FFT, 32.0 * cnt, true);
        launch_k(k_to_dd, nb, 256, 0, s, buf, cnt);
    }
    cdd* r = nullptr;
    nufft_status st = fft_exec<dd>(p, reinterpret_cast<cdd*>(buf), reinterpret_cast<cdd*>(work), batch, dir, s, &r);
    if (st != NUFFT_OK) return st;
    if (cvt_out) {
        Launch L(s, K_FFT, 32.0 * cnt, true);
        launch_k(k_from_dd, nb, 256, 0, s, reinterpret_cast<double2*>(r), cnt);
    }
    NUFFT_CUDA_TRY(cudaGetLastError());
    *result = reinterpret_cast<double2*>(r);
    return NUFFT_OK;
}
template nufft_status fft_exec<double>(const FFTPlan&, double2*, double2*, int64_t, int, cudaStream_t, double2**);

}  // namespace nufft45

// Test hook (not part of the public header): one kernel whose bounded wait
// on a barrier phase that never completes gives up after about a second; the
// next nufft_stream_check reports NUFFT_ERR_TIMEOUT.  Asynchronous on `stream`.
extern "C" nufft_status nufft_debug_wait_expiry(nufft_stream_t stream) {
    using namespace nufft45;
    k_debug_wait_expiry<<<1, 32, 0, (cudaStream_t)stream>>>();
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

// Power-of-two Stockham pass with compile-time radix R = R1 * R2.
//
// Same pass semantics as the generic kernel: for every butterfly j < n/R the
// inputs x[j + k n/R] are twiddled by W_{Ns R}^{(j mod Ns) k}, transformed by
// a length-R DFT and written to y[(j/Ns) Ns R + (j mod Ns) + m Ns].  A CTA
// owns C butterflies.  The length-R DFT is a two-step (four-step) split:
//   step A: each thread (c, k2) holds the R1 inputs k = k1 R2 + k2 in
//           registers, does a register DFT over k1 and multiplies by the
//           inner twiddle W_R^{m1 k2};
//   step B: each thread (c, m1) holds the R2 values (m1, k2) and does a
//           register DFT over k2, giving X[m1 + R1 m2].
// Global loads and stores are staged through shared memory with a mapping
// that keeps every warp access to contiguous addresses; the shared layouts
// are padded so that the transposes are free of bank conflicts.  All index
// arithmetic is shifts and masks.
#pragma once
#include "common.cuh"
#include "df.cuh"

namespace nufft45 {
namespace p2 {

// cos(2 pi k / 32), k = 0..8 (a switch so that constant k folds to a literal)
__device__ __forceinline__ double kC32(int k) {
    switch (k) {
        case 0: return 1.0;
        case 1: return 0.98078528040323044913;
        case 2: return 0.92387953251128675613;
        case 3: return 0.83146961230254523708;
        case 4: return 0.70710678118654752440;
        case 5: return 0.55557023301960222474;
        case 6: return 0.38268343236508977173;
        case 7: return 0.19509032201612826785;
        default: return 0.0;
    }
}

// e^{dir j 2 pi e / 32} for 0 <= e < 16 (compile-time e after unrolling)
template <typename T>
__device__ __forceinline__ c2<T> w32(int e, int dir) {
    T c, s;
    if (e <= 8) { c = (T)kC32(e); s = (T)kC32(8 - e); }
    else { c = -(T)kC32(16 - e); s = (T)kC32(e - 8); }
    return mk<T>(c, dir < 0 ? -s : s);
}

template <int R> struct Log2 { static constexpr int v = 1 + Log2<R / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

__host__ __device__ constexpr int bitrev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

// in-place register DFT of length R (power of two, R <= 32), natural order in
// and out, sum_k v_k e^{dir j 2 pi k m / R}
template <int R, typename T>
__device__ __forceinline__ void dft_reg(c2<T>* v, int dir) {
    if constexpr (R == 1) {
        return;
    } else {
#pragma unroll
        for (int len = R; len >= 2; len >>= 1) {
            const int half = len >> 1;
#pragma unroll
            for (int i = 0; i < R; i += len) {
#pragma unroll
                for (int j = 0; j < half; ++j) {
                    const c2<T> a = v[i + j], b = v[i + j + half];
                    v[i + j] = cadd(a, b);
                    c2<T> d = csub(a, b);
                    const int e = j * (32 / len);
                    if (e == 0) {
                    } else if (e == 8) {
                        d = cmulj(d, dir);
                    } else {
                        d = cmul(d, w32<T>(e, dir));
                    }
                    v[i + j + half] = d;
                }
            }
        }
        // outputs are in bit-reversed order: permute (compile-time)
        c2<T> t[R];
#pragma unroll
        for (int k = 0; k < R; ++k) t[k] = v[k];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = t[bitrev(k, Log2<R>::v)];
    }
}

struct Args {
    int n_log, R_log, Ns_log;  // n = 2^n_log, R = 2^R_log, Ns = 2^Ns_log
    int C_log;                 // C = 2^C_log butterflies per CTA
    int total;                 // batch * n / R butterflies
    int shift;                 // two-level twiddle table split
    const void* tw_full;       // W_n^e for all e < n, or null (then the two-level table)
    // fused element-wise work on the first pass's loads and the last pass's
    // stores, indexed by the element's position idx in its length-n vector:
    //   lop 1: x = src[b * src_bs + ((idx - K0) mod ns)] * fac_in[idx]  (a
    //          deconvolved, scaled selection from an oversampled spectrum)
    //   lop 2: x = in[idx] * fac_in[idx];
    //   sop 1: y *= mulc[idx];  sop 2: y *= fac_out[idx]
    int lop, sop;
    const void* src;
    int64_t src_bs, ns, K0;
    const void* fac_in;
    const void* mulc;
    const void* fac_out;
    // scattering stores (sop 3, 4; TMA-fed pass only): batch stride of the
    // destination, index offset and length
    int64_t out_bs, sel_off, sel_len;
};

template <typename T>
__device__ __forceinline__ c2<T> tw2(const c2<T>* __restrict__ lo, const c2<T>* __restrict__ hi, int shift,
                                     uint32_t e, int dir) {
    c2<T> w = cmul(ldg(&lo[e & ((1u << shift) - 1)]), ldg(&hi[e >> shift]));
    if (dir > 0) w.y = -w.y;
    return w;
}

// W_n^e from the full table when there is one (one load), else two-level
template <typename T>
__device__ __forceinline__ c2<T> twn(const Args& a, const c2<T>* __restrict__ lo, const c2<T>* __restrict__ hi,
                                     uint32_t e, int dir) {
    if (a.tw_full) {
        c2<T> w = ldg(&static_cast<const c2<T>*>(a.tw_full)[e]);
        if (dir > 0) w.y = -w.y;
        return w;
    }
    return tw2<T>(lo, hi, a.shift, e, dir);
}

// compile-time tile: C butterflies per CTA, C * R2 threads
template <typename T, int R1, int R2> struct Cfg {
    static constexpr int R = R1 * R2;
    static constexpr int kElems = sizeof(T) == 4 ? 4096 : 2048;
    static constexpr int C = (kElems / R < 256 / R2) ? kElems / R : 256 / R2;
    static constexpr int TH = C * R2;
    static constexpr int PR = R1 * (R2 + 1) + 1;   // padded column stride (odd)
    static constexpr int NB = R1 / R2;             // (c, m1) groups per thread in step B
};

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(Cfg<T, R1, R2>::TH) k_fft_p2(const c2<T>* in, c2<T>* out, Args a,
                                                               const c2<T>* __restrict__ lo,
                                                               const c2<T>* __restrict__ hi, int dir) {
    pdl_wait();
    pdl_trigger();
    using G = Cfg<T, R1, R2>;
    constexpr int C = G::C, TH = G::TH, PR = G::PR, NB = G::NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* sm = reinterpret_cast<c2<T>*>(smem_raw);
    const int tid = threadIdx.x;
    const int nR_log = a.n_log - a.R_log;      // log2(n/R)
    const uint32_t nR = 1u << nR_log;
    const uint32_t Ns = 1u << a.Ns_log;
    const int g0 = blockIdx.x * C;             // first butterfly of the CTA
    const int tw_shift = a.n_log - a.Ns_log - a.R_log;   // log2(n / (Ns R))
    const int inner_shift = a.n_log - a.R_log;           // W_R^e = W_n^{e n/R}

    // ---- step A: thread (c, k2) holds k = k1 R2 + k2, k1 < R1 ----
    const int ca = tid % C, k2 = tid / C;
    c2<T> v[R1];
    if (nR >= (uint32_t)C) {
        // direct loads: for fixed k1 a warp reads runs of C consecutive butterflies
        const int g = g0 + ca;
        const bool ok = g < a.total;
        const uint32_t b = (uint32_t)g >> nR_log, j = (uint32_t)g & (nR - 1);
        if (a.lop == 1) {
            const c2<T>* gsrc = static_cast<const c2<T>*>(a.src) + (size_t)b * a.src_bs;
            const T* fac = static_cast<const T*>(a.fac_in);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) {
                const int64_t idx = (int64_t)j + ((int64_t)(k1 * R2 + k2) << nR_log);
                int64_t si = idx - a.K0;
                si = si < 0 ? si + a.ns : si;
                v[k1] = ok ? cscale(gsrc[si], ldg(&fac[idx])) : mk<T>(0, 0);
            }
        } else {
            const c2<T>* src = in + ((size_t)b << a.n_log) + j;
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1)
                v[k1] = ok ? src[(size_t)(k1 * R2 + k2) << nR_log] : mk<T>(0, 0);
            if (a.lop == 2) {
                const T* fac = static_cast<const T*>(a.fac_in) + j;
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) v[k1] = cscale(v[k1], ldg(&fac[(size_t)(k1 * R2 + k2) << nR_log]));
            }
        }
        const uint32_t jm = j & (Ns - 1);
        if (jm != 0) {
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) {
                const uint32_t k = (uint32_t)(k1 * R2 + k2);
                if (k != 0) v[k1] = cmul(v[k1], twn<T>(a, lo, hi, (jm * k) << tw_shift, dir));
            }
        }
    } else {
        // several short transforms per CTA (n/R < C, single pass, Ns = 1): the
        // CTA's inputs are one contiguous block; stage it through shared memory
        const int base_b = g0 >> nR_log;   // g0 is a multiple of n/R here
#pragma unroll
        for (int i = 0; i < R1; ++i) {
            const int e = tid + i * TH;
            const int bl = e >> a.n_log, idx = e & ((1 << a.n_log) - 1);
            const int c = (bl << nR_log) + (idx & (nR - 1));
            const int k = idx >> nR_log;
            const bool ok = g0 + c < a.total;
            const c2<T> x = ok ? in[((size_t)(base_b + bl) << a.n_log) + idx] : mk<T>(0, 0);
            sm[c * PR + (k / R2) * (R2 + 1) + (k % R2)] = x;
        }
        __syncthreads();
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = sm[ca * PR + k1 * (R2 + 1) + k2];
        __syncthreads();
    }
    dft_reg<R1, T>(v, dir);
    if (k2 != 0) {
#pragma unroll
        for (int m1 = 1; m1 < R1; ++m1)
            v[m1] = cmul(v[m1], twn<T>(a, lo, hi, (uint32_t)(m1 * k2) << inner_shift, dir));
    }
    {
        c2<T>* col = sm + ca * PR + k2;
#pragma unroll
        for (int m1 = 0; m1 < R1; ++m1) col[m1 * (R2 + 1)] = v[m1];
    }
    __syncthreads();

    // ---- step B: thread (c, m1) -> X[m1 + R1 m2], m2 < R2 ----
    c2<T> w[NB][R2];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const int t = tid + q * TH;
        const int c = t % C, m1 = t / C;
        const c2<T>* row = sm + c * PR + m1 * (R2 + 1);
#pragma unroll
        for (int kk = 0; kk < R2; ++kk) w[q][kk] = row[kk];
        dft_reg<R2, T>(w[q], dir);
    }
    if (Ns >= (uint32_t)C) {
        // direct stores: for fixed m a warp writes runs of C consecutive butterflies
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int t = tid + q * TH;
            const int c = t % C, m1 = t / C;
            const int g = g0 + c;
            if (g < a.total) {
                const uint32_t b = (uint32_t)g >> nR_log, j = (uint32_t)g & (nR - 1);
                const size_t o0 = ((size_t)(j >> a.Ns_log) << (a.Ns_log + a.R_log)) + (j & (Ns - 1));
                c2<T>* dst = out + ((size_t)b << a.n_log) + o0;
                if (a.sop == 1) {
                    const c2<T>* mc = static_cast<const c2<T>*>(a.mulc) + o0;
#pragma unroll
                    for (int m2 = 0; m2 < R2; ++m2) {
                        const size_t o = (size_t)(m1 + R1 * m2) << a.Ns_log;
                        dst[o] = cmul(w[q][m2], ldg(&mc[o]));
                    }
                } else if (a.sop == 2) {
                    const T* fo = static_cast<const T*>(a.fac_out) + o0;
#pragma unroll
                    for (int m2 = 0; m2 < R2; ++m2) {
                        const size_t o = (size_t)(m1 + R1 * m2) << a.Ns_log;
                        dst[o] = cscale(w[q][m2], ldg(&fo[o]));
                    }
                } else {
#pragma unroll
                    for (int m2 = 0; m2 < R2; ++m2) dst[(size_t)(m1 + R1 * m2) << a.Ns_log] = w[q][m2];
                }
            }
        }
    } else {
        // the CTA's outputs form one contiguous block: stage through shared memory
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int t = tid + q * TH;
            const int c = t % C, m1 = t / C;
            c2<T>* col = sm + c * PR + m1;
#pragma unroll
            for (int m2 = 0; m2 < R2; ++m2) col[m2 * R1] = w[q][m2];
        }
        __syncthreads();
        const int g = g0;   // block start: offset e = blk (Ns R) + m Ns + jj, c = blk Ns + jj
        const uint32_t b0 = (uint32_t)g >> nR_log, j0 = (uint32_t)g & (nR - 1);
        const size_t base = ((size_t)b0 << a.n_log) + ((size_t)(j0 >> a.Ns_log) << (a.Ns_log + a.R_log));
#pragma unroll
        for (int i = 0; i < R1; ++i) {
            const int e = tid + i * TH;
            const int blk = e >> (a.Ns_log + a.R_log);
            const int rem = e & ((1 << (a.Ns_log + a.R_log)) - 1);
            const int m = rem >> a.Ns_log;
            const int c = (blk << a.Ns_log) + (rem & (Ns - 1));
            if (g0 + c < a.total) out[base + e] = sm[c * PR + m];
        }
    }
}

}  // namespace p2
}  // namespace nufft45

namespace nufft45 {
namespace p2 {

// ---- streaming variant for multi-pass plans (n/R >= C) ----------------------
// A grid of a few CTAs per SM walks over the tiles of C butterflies; while a
// tile is transformed, the next one is fetched into the other half of a
// double buffer with cp.async (global -> shared, no registers).  The shared
// tile is [k][c] (c contiguous); both register-DFT steps read rows of C
// consecutive columns with the thread's column index fastest, so neither needs
// padding.  Twiddles come from a single table of W_n (one load each).

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T, int R1, int R2> struct SCfg {
    static constexpr int R = R1 * R2;
    static constexpr int kElems = sizeof(T) == 4 ? 4096 : 2048;
    static constexpr int C = (kElems / R < 256 / R2) ? kElems / R : 256 / R2;
    static constexpr int TH = C * R2;
    static constexpr int NB = R1 / R2;
    static constexpr int EPC = 16 / (int)sizeof(c2<T>);   // elements per 16-byte copy
    // resident CTAs per SM the register budget must allow (shared memory
    // holds two tiles of C*R elements: 64 KB for float, 64 KB for double)
    static constexpr int kMinBlocks = (TH >= 256) ? 3 : 4;
};

struct SArgs {
    int n_log, R_log, Ns_log;
    int ntiles;          // batch * n / R / C
    // double-float passes only: the input holds float64 pairs (converted on
    // load) / the output is written as float64 pairs
    int cvt_in, cvt_out;
};

// element load / store with an optional float64 <-> double-float conversion;
// a complex double-float has the size of a double2, so a buffer can hold either
template <typename T> __device__ __forceinline__ c2<T> ld_cvt(const c2<T>* p, int) { return *p; }
template <> __device__ __forceinline__ cdd ld_cvt<dd>(const cdd* p, int cvt) {
    if (!cvt) return *p;
    const double2 d = *reinterpret_cast<const double2*>(p);
    cdd r;
    r.x = dd_from_double(d.x);
    r.y = dd_from_double(d.y);
    return r;
}
template <typename T> __device__ __forceinline__ void st_cvt(c2<T>* p, const c2<T>& v, int) { *p = v; }
template <> __device__ __forceinline__ void st_cvt<dd>(cdd* p, const cdd& v, int cvt) {
    if (cvt) *reinterpret_cast<double2*>(p) = make_double2(dd_to_double(v.x), dd_to_double(v.y));
    else *p = v;
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void s_issue(const c2<T>* __restrict__ in, c2<T>* stage, int tile, const SArgs& a) {
    using G = SCfg<T, R1, R2>;
    constexpr int C = G::C, R = G::R, EPC = G::EPC;
    const int nR_log = a.n_log - a.R_log;
    const int g0 = tile * C;
    const uint32_t b = (uint32_t)g0 >> nR_log, j0 = (uint32_t)g0 & ((1u << nR_log) - 1);
    const c2<T>* src = in + ((size_t)b << a.n_log) + j0;
    constexpr int CP = C / EPC;                 // 16-byte copies per row
    constexpr int ITER = R * CP / G::TH;        // copies per thread (exact)
#pragma unroll
    for (int i = 0; i < ITER; ++i) {
        const int e = threadIdx.x + i * G::TH;
        const int k = e / CP, cc = (e % CP) * EPC;
        cp_async16(stage + k * C + cc, src + ((size_t)k << nR_log) + cc);
    }
}

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(SCfg<T, R1, R2>::TH, SCfg<T, R1, R2>::kMinBlocks) k_fft_p2s(const c2<T>* __restrict__ in,
                                                                 c2<T>* __restrict__ out, SArgs a,
                                                                 const c2<T>* __restrict__ tw, int dir) {
    pdl_wait();
    pdl_trigger();
    using G = SCfg<T, R1, R2>;
    constexpr int R = G::R, C = G::C, NB = G::NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* stage0 = reinterpret_cast<c2<T>*>(smem_raw);
    c2<T>* stage1 = stage0 + R * C;
    const int tid = threadIdx.x;
    const int nR_log = a.n_log - a.R_log;
    const uint32_t nR = 1u << nR_log;
    const uint32_t Ns = 1u << a.Ns_log;
    const int tw_shift = a.n_log - a.Ns_log - a.R_log;
    const int inner_shift = a.n_log - a.R_log;
    const int ca = tid % C, k2 = tid / C;       // step A thread
    int tile = blockIdx.x;
    if (tile >= a.ntiles) return;
    s_issue<T, R1, R2>(in, stage0, tile, a);
    cp_async_commit();
    int buf = 0;
    for (; tile < a.ntiles; tile += gridDim.x, buf ^= 1) {
        c2<T>* st = buf ? stage1 : stage0;
        const int next = tile + gridDim.x;
        if (next < a.ntiles) s_issue<T, R1, R2>(in, buf ? stage0 : stage1, next, a);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int g0 = tile * C;
        // step A: k = k1 R2 + k2 for column ca, pass twiddle, DFT over k1, inner twiddle
        {
            const uint32_t j = ((uint32_t)(g0 + ca)) & (nR - 1);
            const uint32_t jm = j & (Ns - 1);
            c2<T> v[R1];
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) {
                const int k = k1 * R2 + k2;
                c2<T> x = ld_cvt<T>(&st[k * C + ca], a.cvt_in);
                if (jm != 0 && k != 0) {
                    c2<T> w = ldg(&tw[(jm * (uint32_t)k) << tw_shift]);
                    if (dir > 0) w.y = -w.y;
                    x = cmul(x, w);
                }
                v[k1] = x;
            }
            dft_reg<R1, T>(v, dir);
            if (k2 != 0) {
#pragma unroll
                for (int m1 = 1; m1 < R1; ++m1) {
                    c2<T> w = ldg(&tw[(uint32_t)(m1 * k2) << inner_shift]);
                    if (dir > 0) w.y = -w.y;
                    v[m1] = cmul(v[m1], w);
                }
            }
#pragma unroll
            for (int m1 = 0; m1 < R1; ++m1) st[(m1 * R2 + k2) * C + ca] = v[m1];
        }
        __syncthreads();
        // step B: (c, m1) -> X[m1 + R1 m2]
        c2<T> w2[NB][R2];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int t = tid + q * G::TH;
            const int c = t % C, m1 = t / C;
#pragma unroll
            for (int kk = 0; kk < R2; ++kk) w2[q][kk] = st[(m1 * R2 + kk) * C + c];
            dft_reg<R2, T>(w2[q], dir);
        }
        if (Ns >= (uint32_t)C) {
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int t = tid + q * G::TH;
                const int c = t % C, m1 = t / C;
                const uint32_t g = (uint32_t)(g0 + c);
                const uint32_t b = g >> nR_log, j = g & (nR - 1);
                c2<T>* dst = out + ((size_t)b << a.n_log) + ((size_t)(j >> a.Ns_log) << (a.Ns_log + a.R_log)) +
                             (j & (Ns - 1));
#pragma unroll
                for (int m2 = 0; m2 < R2; ++m2) st_cvt<T>(&dst[(size_t)(m1 + R1 * m2) << a.Ns_log], w2[q][m2], a.cvt_out);
            }
        } else {
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int t = tid + q * G::TH;
                const int c = t % C, m1 = t / C;
#pragma unroll
                for (int m2 = 0; m2 < R2; ++m2) st[(m1 + R1 * m2) * C + c] = w2[q][m2];
            }
            __syncthreads();
            const uint32_t b0 = (uint32_t)g0 >> nR_log, j0 = (uint32_t)g0 & (nR - 1);
            const size_t base = ((size_t)b0 << a.n_log) + ((size_t)(j0 >> a.Ns_log) << (a.Ns_log + a.R_log));
#pragma unroll
            for (int i = 0; i < R1; ++i) {
                const int e = tid + i * G::TH;
                const int blk = e >> (a.Ns_log + a.R_log);
                const int rem = e & ((1 << (a.Ns_log + a.R_log)) - 1);
                const int m = rem >> a.Ns_log;
                const int c = (blk << a.Ns_log) + (rem & (Ns - 1));
                st_cvt<T>(&out[base + e], st[m * C + c], a.cvt_out);
            }
        }
        __syncthreads();
    }
}

}  // namespace p2
}  // namespace nufft45

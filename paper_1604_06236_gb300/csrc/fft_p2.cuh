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
};

template <typename T>
__device__ __forceinline__ c2<T> tw2(const c2<T>* __restrict__ lo, const c2<T>* __restrict__ hi, int shift,
                                     uint32_t e, int dir) {
    c2<T> w = cmul(__ldg(&lo[e & ((1u << shift) - 1)]), __ldg(&hi[e >> shift]));
    if (dir > 0) w.y = -w.y;
    return w;
}

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) k_fft_p2(const c2<T>* in, c2<T>* out, Args a, const c2<T>* __restrict__ lo,
                                                const c2<T>* __restrict__ hi, int dir) {
    constexpr int R = R1 * R2;
    constexpr int PR = R1 * (R2 + 1) + 1;      // padded column stride (odd)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* sm = reinterpret_cast<c2<T>*>(smem_raw);
    const int C = 1 << a.C_log;
    const int tid = threadIdx.x;
    const int nR_log = a.n_log - a.R_log;      // log2(n/R)
    const uint32_t nR = 1u << nR_log;
    const uint32_t Ns = 1u << a.Ns_log;
    const int g0 = blockIdx.x << a.C_log;      // first butterfly of the CTA
    const int tot = C * R;
    // ---- load (coalesced) + pass twiddle ----
    const bool in_cfast = nR >= (uint32_t)C;
    const int tw_shift = a.n_log - a.Ns_log - a.R_log;   // log2(n / (Ns R))
    for (int e = tid; e < tot; e += blockDim.x) {
        int c, k;
        if (in_cfast) { c = e & (C - 1); k = e >> a.C_log; }
        else {
            const int bl = e >> a.n_log, idx = e & ((1 << a.n_log) - 1);
            c = (bl << nR_log) + (idx & (nR - 1));
            k = idx >> nR_log;
        }
        const int g = g0 + c;
        c2<T> x = mk<T>(0, 0);
        if (g < a.total) {
            const uint32_t b = (uint32_t)g >> nR_log, j = (uint32_t)g & (nR - 1);
            x = in[((size_t)b << a.n_log) + j + ((size_t)k << nR_log)];
            const uint32_t jm = j & (Ns - 1);
            if (jm != 0 && k != 0) x = cmul(x, tw2<T>(lo, hi, a.shift, (jm * (uint32_t)k) << tw_shift, dir));
        }
        const int k1 = k / R2, k2 = k % R2;
        sm[c * PR + k1 * (R2 + 1) + k2] = x;
    }
    __syncthreads();
    // ---- step A: DFT over k1 for each (c, k2), times W_R^{m1 k2} ----
    const int inner_shift = a.n_log - a.R_log;   // W_R^e = W_n^{e n/R}
    for (int t = tid; t < C * R2; t += blockDim.x) {
        const int c = t / R2, k2 = t % R2;
        c2<T> v[R1];
        c2<T>* col = sm + c * PR + k2;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = col[k1 * (R2 + 1)];
        dft_reg<R1, T>(v, dir);
        if (k2 != 0) {
#pragma unroll
            for (int m1 = 1; m1 < R1; ++m1) v[m1] = cmul(v[m1], tw2<T>(lo, hi, a.shift, (uint32_t)(m1 * k2) << inner_shift, dir));
        }
#pragma unroll
        for (int m1 = 0; m1 < R1; ++m1) col[m1 * (R2 + 1)] = v[m1];
    }
    __syncthreads();
    // ---- step B: DFT over k2 for each (c, m1) -> X[m1 + R1 m2] ----
    constexpr int NB = R1 >= R2 ? R1 / R2 : 1;     // (c, m1) groups per thread
    c2<T> v[NB][R2];
    int cc[NB], mm[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const int t = tid + q * blockDim.x;
        cc[q] = -1;
        if (t < C * R1) {
            const int c = t / R1, m1 = t % R1;
            cc[q] = c; mm[q] = m1;
            const c2<T>* row = sm + c * PR + m1 * (R2 + 1);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) v[q][k2] = row[k2];
            dft_reg<R2, T>(v[q], dir);
        }
    }
    // more (c, m1) pairs than threads * NB cannot happen: blockDim = C * R2
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        if (cc[q] >= 0) {
            c2<T>* col = sm + cc[q] * PR + mm[q];
#pragma unroll
            for (int m2 = 0; m2 < R2; ++m2) col[m2 * R1] = v[q][m2];
        }
    }
    __syncthreads();
    // ---- store (coalesced) ----
    const bool out_cfast = Ns >= (uint32_t)C;
    for (int e = tid; e < tot; e += blockDim.x) {
        int c, m;
        if (out_cfast) { c = e & (C - 1); m = e >> a.C_log; }
        else {
            // contiguous region: offset e = blk (Ns R) + m Ns + jj, c = blk Ns + jj
            const int blk = e >> (a.Ns_log + a.R_log);
            const int rem = e & ((1 << (a.Ns_log + a.R_log)) - 1);
            m = rem >> a.Ns_log;
            c = (blk << a.Ns_log) + (rem & (Ns - 1));
        }
        const int g = g0 + c;
        if (g >= a.total) continue;
        const uint32_t b = (uint32_t)g >> nR_log, j = (uint32_t)g & (nR - 1);
        const uint32_t jm = j & (Ns - 1);
        out[((size_t)b << a.n_log) + ((j >> a.Ns_log) << (a.Ns_log + a.R_log)) + jm + ((size_t)m << a.Ns_log)] =
            sm[c * PR + m];
    }
}

}  // namespace p2
}  // namespace nufft45

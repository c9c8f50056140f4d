// Double-float Stockham passes for transforms of few vectors (the plan's
// float64-class FFTs: 1 to eta vectors of 64K-128K points).  Such a pass is
// bound by the latency of each thread's chain of double-float operations, not
// by bandwidth or issue rate, so this kernel gives every length-R sub-transform
// R/4 threads: the R inputs of a column are staged in shared memory and
// transformed there by radix-4 Stockham stages (one radix-2 stage when R is an
// odd power of two), four elements per thread per stage.  With R up to 1024 a
// 64K-point transform takes two passes instead of three radix-64 passes, and
// twice as many threads share the work of each pass.  Batches of many vectors
// (the all-float64 path) gain from the saved pass as well.
//
// Pass layout (the same as the other power-of-two passes): for j < n/R the R
// inputs x[j + k n/R] are twiddled by W_{Ns R}^{(j mod Ns) k}, transformed, and
// written to y[(j/Ns) Ns R + (j mod Ns) + m Ns].  Each CTA takes C = 2
// consecutive columns, so every global access moves a whole 32-byte sector.
#pragma once
#include "df.cuh"
#include "fft_p2.cuh"

namespace nufft45 {
namespace ddq {

struct QArgs {
    int n_log, Ns_log;   // n = 2^n_log, Ns = 2^Ns_log (product of the earlier radices)
    int cvt_in;          // the input holds float64 pairs (first pass)
    int cvt_out;         // write float64 pairs (last pass)
};

constexpr int kCols = 2;

template <int RL>
__global__ void __launch_bounds__(kCols * (1 << RL) / 4) k_fft_ddq(const cdd* __restrict__ in, cdd* __restrict__ out,
                                                                    QArgs a, const cdd* __restrict__ tw, int dir) {
    pdl_wait();
    pdl_trigger();
    constexpr int R = 1 << RL, TPC = R / 4, C = kCols, TH = C * TPC;
    __shared__ __align__(16) cdd sm[C * R];
    __shared__ __align__(16) cdd tws[R];                 // W_R^i, i < R, for the stages
    const int tid = threadIdx.x;
    const int nR_log = a.n_log - RL;
    const uint32_t nR = 1u << nR_log;
    const uint32_t Ns = 1u << a.Ns_log;
    const int64_t g0 = (int64_t)blockIdx.x * C;           // first column over the whole batch
    const int64_t b = g0 >> nR_log;
    const uint32_t j0 = (uint32_t)(g0 & (nR - 1));
    const cdd* src = in + (b << a.n_log);
    cdd* dst = out + (b << a.n_log);
    const int tw_pass = a.n_log - a.Ns_log - RL;

    // the stages' twiddles W_R^i = W_n^{i n/R}, fetched alongside the data
#pragma unroll
    for (int i = 0; i < R / TH; ++i) tws[tid + i * TH] = tw[(uint32_t)(tid + i * TH) << (a.n_log - RL)];
    // load the C columns (C consecutive elements per row), inter-pass twiddle
#pragma unroll
    for (int i = 0; i < R * C / TH; ++i) {
        const int e = tid + i * TH;
        const int c = e % C, k = e / C;
        const uint32_t j = j0 + c;
        cdd x = p2::ld_cvt<dd>(&src[j + ((size_t)k << nR_log)], a.cvt_in);
        const uint32_t jm = j & (Ns - 1);
        if (jm != 0 && k != 0) {
            cdd w = tw[(jm * (uint32_t)k) << tw_pass];
            if (dir > 0) w.y = -w.y;
            x = cmul(x, w);
        }
        sm[c * R + k] = x;
    }
    __syncthreads();

    // radix-4 Stockham stages inside each column: with the stage's block
    // length s, thread t reads col[t + q R/4], q < 4, twiddles by
    // W_{4s}^{(t mod s) q}, and writes col[(t - t mod s) 4 + t mod s + m s]
    // (a rolled loop: each SM runs these stages once or twice per launch, so a
    // fully unrolled body would be fetched cold from the instruction cache)
    const int c = tid / TPC, t = tid % TPC;
    cdd* col = sm + c * R;
#pragma unroll 1
    for (int sl = 0; 2 * sl + 2 <= RL; ++sl) {
        const int s = 1 << (2 * sl);
        const int tm = t & (s - 1);
        cdd v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = col[t + q * TPC];
        if (tm != 0) {
            // W_{4s}^{tm q} = W_R^{tm q R/(4s)}
            const int sh = RL - (2 * sl + 2);
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                cdd w = tws[(tm * q) << sh];
                if (dir > 0) w.y = -w.y;
                v[q] = cmul(v[q], w);
            }
        }
        p2::dft_reg<4, dd>(v, dir);
        __syncthreads();
        const int o = (t - tm) * 4 + tm;
#pragma unroll
        for (int m = 0; m < 4; ++m) col[o + m * s] = v[m];
        __syncthreads();
    }
    if constexpr (RL & 1) {
        // last stage, radix 2 with s = R/2: butterfly u reads and writes
        // col[u] and col[u + R/2] (twiddle W_R^u on the second input)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int u = t + h * TPC;
            cdd x0 = col[u], x1 = col[u + R / 2];
            if (u != 0) {
                cdd w = tws[u];
                if (dir > 0) w.y = -w.y;
                x1 = cmul(x1, w);
            }
            col[u] = cadd(x0, x1);
            col[u + R / 2] = csub(x0, x1);
        }
        __syncthreads();
    }

    // store: y[(j/Ns) Ns R + (j mod Ns) + m Ns]; with Ns >= C the C columns
    // are adjacent in every output row, with Ns = 1 each column is contiguous
    if (Ns >= (uint32_t)C) {
#pragma unroll
        for (int i = 0; i < R * C / TH; ++i) {
            const int e = tid + i * TH;
            const int cc = e % C, m = e / C;
            const uint32_t j = j0 + cc;
            const size_t o = (size_t)(j & ~(Ns - 1)) * R + (j & (Ns - 1)) + (size_t)m * Ns;
            p2::st_cvt<dd>(&dst[o], sm[cc * R + m], a.cvt_out);
        }
    } else {
#pragma unroll
        for (int i = 0; i < R * C / TH; ++i) {
            const int e = tid + i * TH;
            const int m = e % R, cc = e / R;
            const uint32_t j = j0 + cc;
            const size_t o = (size_t)(j & ~(Ns - 1)) * R + (j & (Ns - 1)) + (size_t)m * Ns;
            p2::st_cvt<dd>(&dst[o], sm[cc * R + m], a.cvt_out);
        }
    }
}

}  // namespace ddq
}  // namespace nufft45

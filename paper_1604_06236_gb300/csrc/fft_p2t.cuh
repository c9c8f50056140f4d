// Persistent power-of-two Stockham pass fed by the tensor memory accelerator.
//
// Same pass semantics as k_fft_p2 (fft_p2.cuh): for every butterfly j < n/R
// the inputs x[j + k n/R] are twiddled by W_{Ns R}^{(j mod Ns) k}, transformed
// by a length-R DFT and written to y[(j/Ns) Ns R + (j mod Ns) + m Ns].  A tile
// is C consecutive butterflies of one vector; its C x R inputs form one 4-D
// box (j, k2, k1, vector) of the array, so a single TMA instruction moves it
// into shared memory as [k][c] (c fastest).  A grid of a few CTAs per SM walks
// over the tiles with an S-stage ring: while tile i is transformed, tiles
// i+1 .. i+S-1 are in flight, and stage completion is tracked by mbarrier
// transaction counts instead of per-thread loads.
//
// Each CTA's first tile is its block index; the later ones are handed out by
// per-launch atomic counters, not by block index: when other work on the GPU
// (the next plan's kernels on another stream) holds some of the slots the
// grid was sized for, the CTAs that start late find fewer tiles left instead
// of running their share as a second wave.  The tiles are split into eight
// shards by tile index mod 8, each with its own counter, served by the CTAs
// of the same block index mod 8: one counter for all CTAs made its atomics
// queue (0.5 us more per pass), and more shards balance less.
// Launches take the kTileSlots counter sets in turn (one sequence per
// device), and the last CTA of a launch to finish sets its set back to zero,
// so a launch replayed from a CUDA graph finds it clean; launches kTileSlots
// apart never run at the same time in any stream-ordered use.  The first tile's
// load goes out before any atomic; a CTA takes its next S-1 tiles with one
// atomic, and each later tile by an atomic issued just before the iteration's
// twiddle loads and TMA wait, whose latency it shares (the result is parked
// in shared memory for the refill at the end of the iteration).
//
// Inter-pass twiddles use W^{jm k} = W^{jm k2} W^{jm R2 k1} (k = k1 R2 + k2):
// each thread loads W^{jm k2} and one entry of the per-tile [k1][c] table of
// W^{jm R2 k1}, so a tile of C R elements needs 2 C R / R1 table loads instead
// of C R.  The inner twiddles W_R^{m1 k2} sit in shared memory for the
// lifetime of the CTA.  Every wait is bounded (a poll count and one second):
// on expiry the kernel counts the event in g_wait_expired, drains its copies in
// flight (again with bounded waits) and returns.
//
// FUSE (radix 16 x 16, two-pass length n = R^2 only): the last pass of one
// transform, a pointwise product and the first pass of a second transform of
// the opposite direction in one kernel.  The tile of the last pass (columns j,
// all outputs j + m n/R) holds exactly the inputs j + k n/R of the second
// transform's first-pass butterflies j, and after step B thread (c, m1)
// holds outputs m = m1 + R1 m2, which is the step-A layout (k2 = m1, k1 = m2)
// of that pass: the data never leaves the SM between the two passes.
#pragma once
#include <cuda.h>

#include "fft_p2.cuh"

namespace nufft45 {

constexpr int p2t_tile_slots = 4096;   // tile counter sets of the TMA-fed passes (p2t::kTileSlots)

// number of in-kernel waits that gave up (read and cleared by the host)
__device__ int g_wait_expired;
// per-launch tile counters of the TMA-fed passes (next tile to hand out)
__device__ unsigned g_p2t_tiles[p2t_tile_slots * 8];   // [slot][shard]
__device__ unsigned g_p2t_done[p2t_tile_slots];        // CTAs of the slot's launch that have finished

namespace p2t {

template <int R1, int R2> struct TCfg {
    static constexpr int R = R1 * R2;
    static constexpr int C = (4096 / R < 256 / R2) ? 4096 / R : 256 / R2;   // butterflies per tile
    static constexpr int TH = C * R2;
    static constexpr int NB = R1 / R2;
    static constexpr int TILE = C * R;   // elements per tile (4096)
    static constexpr int TILE_BYTES = TILE * (int)sizeof(float2);
};

constexpr int kStages = 2;      // ring depth
constexpr int kMinBlocks = 3;   // resident CTAs per SM the register budget allows
constexpr int kTileSlots = p2t_tile_slots;          // tile counters, used by launches in turn
constexpr int kPollLimit = 1 << 22;                 // polls of one wait, at most
constexpr unsigned long long kWaitNs = 1000000000;  // and at most one second

struct TArgs {
    int n_log, R_log, Ns_log, C_log;
    int ntiles;
    int slot;             // tile counter of this launch, < kTileSlots
    const float2* fmul;   // FUSE: the pointwise factor between the two transforms (length n)
    // lop 2: x = in[idx] * fac_in[idx]; lop 3 (first pass): the input is zero
    // outside rows k1 < R1/4 and k1 >= 3 R1/4 (a spectrum centred on the
    // grid's index 0 that fills half of it): only those rows are loaded, as two
    // boxes of R1/4 rows, and the others enter the DFT as zeros;
    // sop 1: y *= mulc[idx]; sop 2: y *= fac_out[idx];
    // sop 3: k = (idx + off) mod n, if k < len: out[b out_bs + k] = y fac_out[k];
    // sop 4: out[b out_bs + ((idx - off) mod len)] = y fac_out[idx]
    int lop, sop;
    const float* fac_in;
    const float2* mulc;
    const float* fac_out;
    int64_t out_bs, off, len;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// true once the phase with this parity completed; false after kPollLimit
// polls or kWaitNs nanoseconds, whichever comes first
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (int i = 0; i < kPollLimit; ++i) {
        if (mbar_try_wait(b, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

template <int R1, int R2>
__device__ __forceinline__ void issue(const CUtensorMap* tm, float2* st, uint64_t* bar, int tile, int nR_log,
                                      bool half) {
    using G = TCfg<R1, R2>;
    const int g0 = tile * G::C;
    const int b = g0 >> nR_log, j0 = g0 & ((1 << nR_log) - 1);
    if (half) {
        // rows k1 < R1/4 and k1 >= 3 R1/4 (the tensor map's box is R1/4 rows high)
        mbar_expect_tx(bar, G::TILE_BYTES / 2);
        tma_load_4d(st, tm, bar, j0, 0, 0, b);
        tma_load_4d(st + (3 * R1 / 4) * R2 * G::C, tm, bar, j0, 0, 3 * R1 / 4, b);
    } else {
        mbar_expect_tx(bar, G::TILE_BYTES);
        tma_load_4d(st, tm, bar, j0, 0, 0, b);
    }
}

// staged (Ns = 1) store layout: output m of column c at c R + (m ^ swz(c));
// the XOR keeps both the column-strided writes and the contiguous 16-byte
// reads at the minimum number of shared-memory wavefronts
__device__ __forceinline__ int swz(int c) { return (c & 7) << 1; }

template <int R1, int R2, bool FUSE = false>
__global__ void __launch_bounds__(TCfg<R1, R2>::TH, kMinBlocks)
    k_fft_p2t(const __grid_constant__ CUtensorMap tm, float2* __restrict__ out, TArgs a,
              const float2* __restrict__ tw, int dir) {
    pdl_wait();
    pdl_trigger();
    static_assert(!FUSE || R1 == R2, "the fused pair needs R1 = R2");
    using G = TCfg<R1, R2>;
    constexpr int R = G::R, C = G::C, TH = G::TH, NB = G::NB, TILE = G::TILE, S = kStages;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>(smem_raw);          // S x TILE
    float2* wi = stage + S * TILE;                                 // W_R^e, e < R
    float2* btab = wi + R;                                         // [k1][c]: W^{jm R2 k1}
    uint64_t* bars = reinterpret_cast<uint64_t*>(btab + R1 * C);   // S barriers
    int* tq = reinterpret_cast<int*>(bars + S);                      // tile in each stage, -1: none
    unsigned* tnext = reinterpret_cast<unsigned*>(tq + S);           // counter value for the refill
    const int tid = threadIdx.x;
    const int nR_log = a.n_log - a.R_log;
    const uint32_t nR = 1u << nR_log;
    const uint32_t Ns = 1u << a.Ns_log;
    const int tw_shift = a.n_log - a.Ns_log - a.R_log;
    const int inner_shift = a.n_log - a.R_log;
    const int ntiles = a.ntiles;
    // tiles t = h + nsh u of shard h = blockIdx mod nsh: u < shard_base are
    // the shard's CTAs' first tiles, the later ones come from its counter
    const unsigned nsh = gridDim.x < 8u ? gridDim.x : 8u;
    const unsigned shard = blockIdx.x % nsh;
    const unsigned shard_base = (gridDim.x - shard + nsh - 1u) / nsh;

    for (int e = tid; e < R; e += TH) {
        float2 w = __ldg(&tw[(uint32_t)e << inner_shift]);
        if (dir > 0) w.y = -w.y;
        wi[e] = w;
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // (the grid is at most ntiles CTAs)
        tq[0] = (int)blockIdx.x;
        issue<R1, R2>(&tm, stage, &bars[0], (int)blockIdx.x, nR_log, a.lop == 3);
        const unsigned first = shard_base + atomicAdd(&g_p2t_tiles[a.slot * 8 + shard], (unsigned)(S - 1));
        for (int s = 1; s < S; ++s) {
            const unsigned u = shard + nsh * (first + (unsigned)(s - 1));
            const int t = u < (unsigned)ntiles ? (int)u : -1;
            tq[s] = t;
            if (t >= 0) issue<R1, R2>(&tm, stage + s * TILE, &bars[s], t, nR_log, a.lop == 3);
        }
    }
    __syncthreads();

    const int ca = tid % C, k2 = tid / C;   // step-A thread: column ca, inputs k = k1 R2 + k2
    int it = 0;
    bool expired = false;
    // stages are consumed in the order their tiles were taken, so the first
    // empty one ends the walk (tq[s] was written before a barrier every
    // thread has passed since)
    for (;; ++it) {
        const int s = it % S;
        const int tile = tq[s];
        if (tile < 0) break;
        // the tile this stage loads next (thread 0; parked after the wait below)
        unsigned nxt = 0u;
        if (tid == 0) nxt = atomicAdd(&g_p2t_tiles[a.slot * 8 + shard], 1u);
        float2* st = stage + s * TILE;
        const int g0 = tile * C;
        const uint32_t b = (uint32_t)g0 >> nR_log, j0 = (uint32_t)g0 & (nR - 1);
        float2 wa = make_float2(1.f, 0.f);
        if (a.Ns_log > 0) {
            const uint32_t jm = (j0 + ca) & (Ns - 1);
            wa = __ldg(&tw[(jm * (uint32_t)k2) << tw_shift]);
            if (dir > 0) wa.y = -wa.y;
            for (int e = tid; e < R1 * C; e += TH) {
                const int c = e % C, k1 = e / C;
                const uint32_t jmc = (j0 + c) & (Ns - 1);
                float2 w = __ldg(&tw[(jmc * (uint32_t)(R2 * k1)) << tw_shift]);
                if (dir > 0) w.y = -w.y;
                btab[e] = w;
            }
        }
        const bool ok = mbar_wait(&bars[s], (unsigned)((it / S) & 1));
        if (tid == 0) *tnext = shard + nsh * (shard_base + nxt);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicAdd(&g_wait_expired, 1);
            expired = true;
            break;
        }
        // step A: DFT over k1 of column ca, then the inner twiddle W_R^{m1 k2}
        float2 v[R1];
        const bool half = a.lop == 3;
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            const bool mid = k1 >= R1 / 4 && k1 < 3 * R1 / 4;
            v[k1] = (half && mid) ? make_float2(0.f, 0.f) : st[(k1 * R2 + k2) * C + ca];
        }
        if (a.lop == 2) {
            const float* fac = a.fac_in + j0 + ca;
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) v[k1] = cscale(v[k1], __ldg(&fac[(size_t)(k1 * R2 + k2) << nR_log]));
        }
        if (a.Ns_log > 0) {
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) v[k1] = cmul(v[k1], cmul(wa, btab[k1 * C + ca]));
        }
        p2::dft_reg<R1, float>(v, dir);
        if (k2 != 0) {
#pragma unroll
            for (int m1 = 1; m1 < R1; ++m1) v[m1] = cmul(v[m1], wi[m1 * k2]);
        }
        // in place: this thread's outputs (m1, k2) take the slots of its inputs (k1, k2)
#pragma unroll
        for (int m1 = 0; m1 < R1; ++m1) st[(m1 * R2 + k2) * C + ca] = v[m1];
        __syncthreads();
        // step B: thread (c, m1) -> X[m1 + R1 m2], m2 < R2
        float2 w[NB][R2];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int t = tid + q * TH;
            const int c = t % C, m1 = t / C;
#pragma unroll
            for (int kk = 0; kk < R2; ++kk) w[q][kk] = st[(m1 * R2 + kk) * C + c];
            p2::dft_reg<R2, float>(w[q], dir);
        }
        if constexpr (FUSE) {
            // x fmul at the outputs o = j + m n/R of the finished transform, then
            // the second transform's first pass (direction -dir, Ns = 1) from
            // registers: thread (c, m1) is its step-A thread (ca = c, k2 = m1)
            const float2* fm = a.fmul + (j0 + ca);
            float2 u[R1];
#pragma unroll
            for (int m2 = 0; m2 < R2; ++m2) u[m2] = cmul(w[0][m2], __ldg(&fm[(size_t)(k2 + R1 * m2) << a.Ns_log]));
            p2::dft_reg<R1, float>(u, -dir);
            if (k2 != 0) {
#pragma unroll
                for (int m1 = 1; m1 < R1; ++m1) u[m1] = cmul(u[m1], cconj(wi[m1 * k2]));
            }
            __syncthreads();   // every step-B read of the first transform is done
#pragma unroll
            for (int m1 = 0; m1 < R1; ++m1) st[(m1 * R2 + k2) * C + ca] = u[m1];
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < R2; ++kk) w[0][kk] = st[(k2 * R2 + kk) * C + ca];
            p2::dft_reg<R2, float>(w[0], -dir);
        }
        if (!FUSE && a.Ns_log >= a.C_log) {
            // direct stores: for fixed m a warp writes runs of C consecutive butterflies
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int t = tid + q * TH;
                const int c = t % C, m1 = t / C;
                const uint32_t j = j0 + c;
                const size_t o0 = ((size_t)(j >> a.Ns_log) << (a.Ns_log + a.R_log)) + (j & (Ns - 1));
                float2* dst = out + ((size_t)b << a.n_log) + o0;
                if (a.sop == 3) {
                    const int64_t n = (int64_t)1 << a.n_log;
                    float2* sd = out + (int64_t)b * a.out_bs;
#pragma unroll
                    for (int m2 = 0; m2 < R2; ++m2) {
                        int64_t k = (int64_t)o0 + ((int64_t)(m1 + R1 * m2) << a.Ns_log) + a.off;
                        k = k >= n ? k - n : k;
                        if (k < a.len) sd[k] = cscale(w[q][m2], __ldg(&a.fac_out[k]));
                    }
                } else if (a.sop == 4) {
                    float2* sd = out + (int64_t)b * a.out_bs;
#pragma unroll
                    for (int m2 = 0; m2 < R2; ++m2) {
                        const int64_t o = (int64_t)o0 + ((int64_t)(m1 + R1 * m2) << a.Ns_log);
                        int64_t g = o - a.off;
                        g = g < 0 ? g + a.len : g;
                        sd[g] = cscale(w[q][m2], __ldg(&a.fac_out[o]));
                    }
                } else if (a.sop == 1) {
                    const float2* mc = a.mulc + o0;
#pragma unroll
                    for (int m2 = 0; m2 < R2; ++m2) {
                        const size_t o = (size_t)(m1 + R1 * m2) << a.Ns_log;
                        dst[o] = cmul(w[q][m2], __ldg(&mc[o]));
                    }
                } else if (a.sop == 2) {
                    const float* fo = a.fac_out + o0;
#pragma unroll
                    for (int m2 = 0; m2 < R2; ++m2) {
                        const size_t o = (size_t)(m1 + R1 * m2) << a.Ns_log;
                        dst[o] = cscale(w[q][m2], __ldg(&fo[o]));
                    }
                } else {
#pragma unroll
                    for (int m2 = 0; m2 < R2; ++m2) dst[(size_t)(m1 + R1 * m2) << a.Ns_log] = w[q][m2];
                }
            }
        } else {
            // Ns = 1: the tile's outputs are one contiguous block of C R elements
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int t = tid + q * TH;
                const int c = t % C, m1 = t / C;
#pragma unroll
                for (int m2 = 0; m2 < R2; ++m2) st[c * R + ((m1 + R1 * m2) ^ swz(c))] = w[q][m2];
            }
            __syncthreads();
            float4* dst = reinterpret_cast<float4*>(out + ((size_t)b << a.n_log) + ((size_t)j0 << a.R_log));
            const float4* src = reinterpret_cast<const float4*>(st);
#pragma unroll
            for (int i = 0; i < TILE / 2 / TH; ++i) {
                const int e2 = tid + i * TH;
                const int e = 2 * e2;
                const int c = e / R, m = e % R;
                dst[e2] = src[(c * R + (m ^ swz(c))) >> 1];
            }
        }
        // order this stage's generic-proxy accesses before the TMA refill
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            const unsigned u = *tnext;
            const int t = u < (unsigned)ntiles ? (int)u : -1;
            tq[s] = t;
            if (t >= 0) issue<R1, R2>(&tm, st, &bars[s], t, nR_log, a.lop == 3);
        }
    }
    if (tid == 0) {
        // after an expired wait, let the copies still in flight land before the CTA ends
        if (expired) {
            for (int k = 0; k < S; ++k) {
                const int ss = (it + k) % S;
                if (tq[ss] >= 0) mbar_wait(&bars[ss], (unsigned)(((it + k) / S) & 1));
            }
        }
        // the last CTA to finish leaves the launch's counters at zero (every
        // CTA has taken its last tile before it counts itself done)
        __threadfence();
        if (atomicAdd(&g_p2t_done[a.slot], 1u) == gridDim.x - 1) {
            for (unsigned h = 0; h < 8u; ++h) g_p2t_tiles[a.slot * 8 + h] = 0u;
            g_p2t_done[a.slot] = 0u;
            __threadfence();
        }
    }
}

template <int R1, int R2>
constexpr size_t smem_bytes() {
    using G = TCfg<R1, R2>;
    return (size_t)kStages * G::TILE * sizeof(float2) + (size_t)G::R * sizeof(float2) +
           (size_t)R1 * G::C * sizeof(float2) + kStages * (sizeof(uint64_t) + sizeof(int)) + sizeof(unsigned);
}

}  // namespace p2t
}  // namespace nufft45

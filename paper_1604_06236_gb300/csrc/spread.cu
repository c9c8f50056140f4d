// Node geometry (exact cells, counting sort), output-stationary spreading
// (type-1 gridding) and interpolation (type-2), and the pointwise stages.
//
// Spreading is a gather: every grid point g owns its sum
//     b_g = sum_p c_p phi(g - n t_p),
// and reads the nodes of cells [g - w/2, g + w/2 - 1], a contiguous range of
// the cell-sorted (and periodically extended) node list.  A CTA stages the
// nodes of its tile in shared memory, each thread accumulates its grid
// point(s) in registers for a chunk of right-hand sides, and the tile is
// written once with coalesced stores: no atomics on the grid, deterministic
// summation order.
#include "internal.h"
#include "df.cuh"

#include <algorithm>

namespace nufft45 {

namespace {

constexpr int kTB = 256;

inline unsigned nblk(int64_t n, int tb = kTB) { return (unsigned)((n + tb - 1) / tb); }

// t = x / (2 pi) mod 1 (IEEE division and floor) as exact turns T =
// trunc(t 2^64); cell = floor(n t) = high word of T n and its fraction = low
// word / 2^64, exactly; per-cell counts; per-block sums of T mod 2^64 (unsigned
// wrap-around is exact arithmetic mod 1 in turns); block 0 clears the
// duplicate flag
__global__ void k_node_prep(const double* __restrict__ x, int64_t N, uint64_t n, uint64_t* __restrict__ T,
                            int* __restrict__ cell, double* __restrict__ frac, int* __restrict__ count,
                            unsigned long long* __restrict__ partial, int* __restrict__ dup) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s[kTB];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long t = 0;
    if (i < N) {
        double u = x[i] / 6.283185307179586476925286766559;
        u -= floor(u);
        if (u >= 1.0) u = 0.0;
        t = __double2ull_rz(u * 18446744073709551616.0);
        T[i] = t;
        const int c = (int)__umul64hi(t, n);
        cell[i] = c;
        frac[i] = (double)(t * n) * 5.42101086242752217003726400434970855712890625e-20;
        atomicAdd(&count[c], 1);
    }
    s[threadIdx.x] = t;
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) s[threadIdx.x] += s[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s[0];
        if (blockIdx.x == 0) *dup = 0;
    }
}

// exclusive scan of int counts in two launches: k_scan_blocks scans blocks of
// kScanPer entries (warp shuffles, then the warps' totals) and writes each
// block's total; k_scan_add adds to every entry the totals of the blocks
// before its own.  out has L entries (the caller scans n + 1 counts, the
// last one zero, so out[n] is the total).
constexpr int kScanTB = 1024;
constexpr int kScanPer = 2 * kScanTB;

// (the counts are cleared as they are read: they serve again as fill counters)
__global__ void k_scan_blocks(int* __restrict__ in, int64_t L, int* __restrict__ out, int* __restrict__ sums) {
    pdl_wait();
    pdl_trigger();
    __shared__ int wsum[kScanTB / 32];
    const int64_t i0 = (int64_t)blockIdx.x * kScanPer + 2 * threadIdx.x;
    int a = 0, b = 0;
    if (i0 < L) { a = in[i0]; in[i0] = 0; }
    if (i0 + 1 < L) { b = in[i0 + 1]; in[i0 + 1] = 0; }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = a + b;   // inclusive scan of the pair sums within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    if (lane == 31) wsum[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int u = wsum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, u, d);
            if (lane >= d) u += t;
        }
        wsum[lane] = u;   // inclusive over the warps
    }
    __syncthreads();
    const int base = (wid > 0 ? wsum[wid - 1] : 0) + v - (a + b);   // exclusive, this thread's pair
    if (i0 < L) out[i0] = base;
    if (i0 + 1 < L) out[i0 + 1] = base + a;
    if (threadIdx.x == 0) sums[blockIdx.x] = wsum[kScanTB / 32 - 1];
}

// (block 0 also adds up the per-block turn sums of k_node_prep: sumT)
__global__ void k_scan_add(int* __restrict__ out, int64_t L, const int* __restrict__ sums,
                           const unsigned long long* __restrict__ partial, int64_t np,
                           unsigned long long* __restrict__ sumT) {
    pdl_wait();
    pdl_trigger();
    __shared__ int carry_w[kTB / 32];
    __shared__ unsigned long long r[kTB];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // this block lies inside scan block sb (kScanPer is a multiple of blockDim)
    const int64_t sb = ((int64_t)blockIdx.x * blockDim.x) / kScanPer;
    int c = 0;
    for (int64_t k = threadIdx.x; k < sb; k += blockDim.x) c += sums[k];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0) carry_w[threadIdx.x >> 5] = c;
    if (blockIdx.x == 0) {
        unsigned long long acc = 0;
        for (int64_t k = threadIdx.x; k < np; k += blockDim.x) acc += partial[k];
        r[threadIdx.x] = acc;
    }
    __syncthreads();
    int carry = 0;
#pragma unroll
    for (int w = 0; w < kTB / 32; ++w) carry += carry_w[w];
    if (i < L) out[i] += carry;
    if (blockIdx.x == 0) {
        for (int d = blockDim.x / 2; d > 0; d >>= 1) {
            if (threadIdx.x < d) r[threadIdx.x] += r[threadIdx.x + d];
            __syncthreads();
        }
        if (threadIdx.x == 0) *sumT = r[0];
    }
}

__global__ void k_scatter(const int* __restrict__ cell, int64_t N, const int* __restrict__ start,
                          int* __restrict__ fill, int* __restrict__ perm) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int c = cell[i];
    perm[start[c] + atomicAdd(&fill[c], 1)] = (int)i;
}

// order the nodes of each cell by (T, index): deterministic, and equal nodes
// become neighbours for the duplicate check
__global__ void k_order_cells(const int* __restrict__ start, int64_t n, const uint64_t* __restrict__ T,
                              int* __restrict__ perm) {
    pdl_wait();
    pdl_trigger();
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int a = start[c], b = start[c + 1];
    for (int i = a + 1; i < b; ++i) {
        const int p = perm[i];
        const uint64_t tp = T[p];
        int j = i - 1;
        while (j >= a) {
            const int q = perm[j];
            const uint64_t tq = T[q];
            if (tq < tp || (tq == tp && q < p)) break;
            perm[j + 1] = q;
            --j;
        }
        perm[j + 1] = p;
    }
}

// One launch over three ranges: [0, N) the sorted slots (cell, fraction and
// the coincident-node check: neighbours in sorted, i.e. cyclic turn, order
// closer than 2^-44 turns, including the pair that wraps from the last to the
// first); [N, 3N) the extended list [nodes of cells n-h..n-1, shifted by -n]
// [all nodes] [nodes of cells 0..h-1, shifted by +n], h = w/2; [3N, 3N+n+w+1)
// the extended list's cell starts cstart[e], e = cell + h in [0, n + w]
__global__ void k_fill(const int* __restrict__ start, int64_t n, int w, int64_t N, const int* __restrict__ perm,
                       const int* __restrict__ cell, const double* __restrict__ frac, const uint64_t* __restrict__ T,
                       int* __restrict__ scell, double* __restrict__ sfrac, float* __restrict__ sfracf,
                       int* __restrict__ dup, int* __restrict__ eperm, int* __restrict__ ecell,
                       double* __restrict__ efrac, float* __restrict__ efracf, int* __restrict__ cstart) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int h = w / 2;
    if (i < N) {
        const int p = perm[i];
        scell[i] = cell[p];
        const double f = frac[p];
        sfrac[i] = f;
        if (sfracf) sfracf[i] = (float)f;
        if (N > 1) {
            const uint64_t d = T[perm[i + 1 < N ? i + 1 : 0]] - T[p];
            if (d < (1ull << 20)) *dup = 1;
        }
        return;
    }
    const int pre = start[n] - start[n - h];
    if (i < 3 * N) {
        const int64_t e = i - N;
        const int post = start[h];
        if (e >= pre + N + post) return;
        int64_t slot;
        int shift;
        if (e < pre) { slot = start[n - h] + e; shift = -(int)n; }
        else if (e < pre + N) { slot = e - pre; shift = 0; }
        else { slot = e - pre - N; shift = (int)n; }
        const int p = perm[slot];
        eperm[e] = p;
        ecell[e] = cell[p] + shift;
        const double f = frac[p];
        efrac[e] = f;
        if (efracf) efracf[e] = (float)f;
        return;
    }
    const int64_t e = i - 3 * N;
    if (e > n + w) return;
    int v;
    if (e < h) v = start[n - h + e] - start[n - h];
    else if (e < n + h) v = pre + start[e - h];
    else v = pre + (int)N + start[e - h - n];
    cstart[e] = v;
}

// ---- spreading (gather) -----------------------------------------------------
template <typename T> struct FracPtr;
template <> struct FracPtr<float> { static const float* ext(const Geometry& g) { return g.ext_fracf; } static const float* srt(const Geometry& g) { return g.srt_fracf; } };
template <> struct FracPtr<double> { static const double* ext(const Geometry& g) { return g.ext_frac; } static const double* srt(const Geometry& g) { return g.srt_frac; } };

constexpr int kChunk = 256;

// output-stationary gather: grid point g sums the extended nodes of the
// cells within w/2 of it, BC right-hand sides per block row
template <typename T, int BC>
__global__ void __launch_bounds__(kTB) k_spread(int64_t n, int w, T two_over_w, T beta, const int* __restrict__ cstart,
                                                const int* __restrict__ eperm, const int* __restrict__ ecell,
                                                const T* __restrict__ efrac, const c2<T>* __restrict__ src,
                                                int64_t src_bs, const c2<T>* __restrict__ wt, c2<T>* __restrict__ grid,
                                                int64_t batch) {
    pdl_wait();
    pdl_trigger();
    __shared__ int s_cell[kChunk];
    __shared__ T s_frac[kChunk];
    __shared__ c2<T> s_str[BC][kChunk];
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t g = g0 + threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.y * BC;
    const int64_t glast = min(g0 + (int64_t)blockDim.x, n) - 1;
    const int t0 = cstart[g0], t1 = cstart[glast + w];
    int lo = 0, hi = 0;
    if (g < n) { lo = cstart[g]; hi = cstart[g + w]; }
    c2<T> acc[BC];
#pragma unroll
    for (int b = 0; b < BC; ++b) acc[b] = mk<T>(0, 0);
    for (int ch = t0; ch < t1; ch += kChunk) {
        const int cnt = min(kChunk, t1 - ch);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = ch + e;
            s_cell[e] = ecell[i];
            s_frac[e] = efrac[i];
            const c2<T> wv = wt[i];
            if (src) {
                const int p = eperm[i];
#pragma unroll
                for (int b = 0; b < BC; ++b)
                    s_str[b][e] = (b0 + b < batch) ? cmul(src[(b0 + b) * src_bs + p], wv) : mk<T>(0, 0);
            } else {
#pragma unroll
                for (int b = 0; b < BC; ++b) s_str[b][e] = wv;
            }
        }
        __syncthreads();
        const int a = max(lo, ch), z = min(hi, ch + cnt);
        for (int i = a; i < z; ++i) {
            const int e = i - ch;
            const T d = (T)(int)(g - s_cell[e]) - s_frac[e];   // small offset: a 32-bit integer conversion
            const T ph = es_kernel<T>(d, two_over_w, beta);
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                acc[b].x = fma(ph, s_str[b][e].x, acc[b].x);
                acc[b].y = fma(ph, s_str[b][e].y, acc[b].y);
            }
        }
    }
    if (g < n) {
#pragma unroll
        for (int b = 0; b < BC; ++b)
            if (b0 + b < batch) grid[(b0 + b) * n + g] = acc[b];
    }
}

// ---- float32 spread for many right-hand sides (tiled, pipelined) ----------
// One CTA per tile of kTB grid points, all right-hand sides.  The nodes of
// the tile's window (extended slots t0 .. t1, at most one per thread) are
// read once: each thread tabulates the w kernel values of its node,
// ph[e][m] = phi(m + 1 - w/2 - frac_e) (grid point cell_e + 1 - w/2 + m).
// The samples of a chunk of BC right-hand sides at those nodes are gathered
// into a two-stage ring by cp.async while the previous chunk is summed; once
// a chunk has landed, its node's thread multiplies it by the slot weight, and
// each grid point then sums ph x strength over the nodes of its window in
// registers and is written once per right-hand side.  Tiles whose window
// holds more than kTB nodes (dense clusters) take the window in pieces,
// without the ring.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

constexpr int kTileList = 8;   // a grid point's nodes whose kernel values are listed once per tile

struct TileSmem {
    float* ph;      // [kTB][w]
    float2* ring;   // [2][BC][kTB]
    float2* wt;     // [kTB]
    int* cell;      // [kTB]
    float* kl;      // [kTileList][kTB]: the grid point's kernel values, node by node
};

// node e = threadIdx.x of the piece [c0, c0 + cnt): cell, slot weight and the
// w kernel values; returns its node index (the sample column), -1 if none
__device__ __forceinline__ int tile_tabulate(const TileSmem& sm, int c0, int cnt, int w, float two_over_w, float beta,
                                             const int* __restrict__ eperm, const int* __restrict__ ecell,
                                             const float* __restrict__ efrac, const float2* __restrict__ wt) {
    const int e = threadIdx.x;
    if (e >= cnt) return -1;
    const int h = w / 2;
    sm.cell[e] = ecell[c0 + e];
    sm.wt[e] = wt[c0 + e];
    const float f = efrac[c0 + e];
    float* ph = sm.ph + e * w;
    for (int m = 0; m < w; ++m) ph[m] = es_kernel<float>((float)(m + 1 - h) - f, two_over_w, beta);
    return eperm[c0 + e];
}

// this thread's node's samples of right-hand sides [bc BC, bc BC + BC) into
// ring stage st (one commit group per thread, possibly empty)
template <int BC>
__device__ __forceinline__ void tile_gather(const TileSmem& sm, int bc, int st, int p,
                                            const float2* __restrict__ src, int64_t src_bs, int64_t batch) {
    if (p >= 0) {
        float2* dst = sm.ring + st * BC * kTB + threadIdx.x;
        const int64_t b0 = (int64_t)bc * BC;
        const float2* sp = src + b0 * src_bs + p;
        const int nb = (int)min((int64_t)BC, batch - b0);
#pragma unroll
        for (int b = 0; b < BC; ++b)
            if (b < nb) cp_async8(dst + b * kTB, sp + b * src_bs);
    }
    cp_async_commit();
}

// x slot weight, in place (the thread's own node column)
template <int BC>
__device__ __forceinline__ void tile_weight(const TileSmem& sm, int st, int p) {
    if (p < 0) return;
    float2* col = sm.ring + st * BC * kTB + threadIdx.x;
    const float2 wv = sm.wt[threadIdx.x];
#pragma unroll
    for (int b = 0; b < BC; ++b) col[b * kTB] = cmul(col[b * kTB], wv);
}

template <int BC>
__device__ __forceinline__ void tile_accumulate(const TileSmem& sm, float2* acc, int st, int c0, int a, int z,
                                                int64_t g, int w) {
    const float2* sv = sm.ring + st * BC * kTB;
    const int h = w / 2;
    for (int i = a; i < z; ++i) {
        const int e = i - c0;
        const float k = sm.ph[e * w + (int)(g - sm.cell[e]) - 1 + h];
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            const float2 v = sv[b * kTB + e];
            acc[b].x = fmaf(k, v.x, acc[b].x);
            acc[b].y = fmaf(k, v.y, acc[b].y);
        }
    }
}

// as tile_accumulate for a grid point whose nl <= kTileList nodes (window
// columns e0 .. e0 + nl - 1) have their kernel values listed in sm.kl: the
// same sums in the same order, without the per-chunk cell and tap lookups
template <int BC>
__device__ __forceinline__ void tile_accumulate_list(const TileSmem& sm, float2* acc, int st, int e0, int nl) {
    const float2* sv = sm.ring + st * BC * kTB + e0;
    const float* kl = sm.kl + threadIdx.x;
    for (int j = 0; j < nl; ++j) {
        const float k = kl[j * kTB];
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            const float2 v = sv[b * kTB + j];
            acc[b].x = fmaf(k, v.x, acc[b].x);
            acc[b].y = fmaf(k, v.y, acc[b].y);
        }
    }
}

template <int BC>
__global__ void __launch_bounds__(kTB) k_spread_tile(int64_t n, int w, float two_over_w, float beta,
                                                     const int* __restrict__ cstart, const int* __restrict__ eperm,
                                                     const int* __restrict__ ecell, const float* __restrict__ efrac,
                                                     const float2* __restrict__ src, int64_t src_bs,
                                                     const float2* __restrict__ wt, float2* __restrict__ grid,
                                                     int64_t batch) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem sm;
    sm.ring = reinterpret_cast<float2*>(smem_raw);
    sm.wt = sm.ring + 2 * BC * kTB;
    sm.ph = reinterpret_cast<float*>(sm.wt + kTB);
    sm.cell = reinterpret_cast<int*>(sm.ph + kTB * w);
    sm.kl = reinterpret_cast<float*>(sm.cell + kTB);
    const int64_t g0 = (int64_t)blockIdx.x * kTB;
    const int64_t g = g0 + threadIdx.x;
    const int64_t glast = min(g0 + (int64_t)kTB, n) - 1;
    const int t0 = cstart[g0], t1 = cstart[glast + w];
    int lo = 0, hi = 0;
    if (g < n) { lo = cstart[g]; hi = cstart[g + w]; }
    const int nchunks = (int)((batch + BC - 1) / BC);
    const int cnt_all = t1 - t0;
    float2* out = grid + g;
    float2 acc[BC];
    if (cnt_all <= kTB) {
        const int p = tile_tabulate(sm, t0, cnt_all, w, two_over_w, beta, eperm, ecell, efrac, wt);
        tile_gather<BC>(sm, 0, 0, p, src, src_bs, batch);
        int nl = -1;   // this grid point's listed nodes (-1: too many, looked up per chunk)
        for (int bc = 0; bc < nchunks; ++bc) {
            const int st = bc & 1;
            if (bc + 1 < nchunks) {
                tile_gather<BC>(sm, bc + 1, st ^ 1, p, src, src_bs, batch);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            tile_weight<BC>(sm, st, p);   // the thread's own copies: no barrier needed before
            __syncthreads();
            if (bc == 0 && hi - lo <= kTileList) {
                // the kernel values of this grid point's nodes, once for all chunks
                // (written and read by this thread only)
                const int h = w / 2;
                for (int j = 0; j < hi - lo; ++j) {
                    const int e = lo - t0 + j;
                    sm.kl[j * kTB + threadIdx.x] = sm.ph[e * w + (int)(g - sm.cell[e]) - 1 + h];
                }
                nl = hi - lo;
            }
#pragma unroll
            for (int b = 0; b < BC; ++b) acc[b] = make_float2(0.f, 0.f);
            if (nl >= 0) tile_accumulate_list<BC>(sm, acc, st, lo - t0, nl);
            else tile_accumulate<BC>(sm, acc, st, t0, lo, hi, g, w);
            if (g < n) {
                const int nb = (int)min((int64_t)BC, batch - (int64_t)bc * BC);
                float2* o = out + (int64_t)bc * BC * n;
#pragma unroll
                for (int b = 0; b < BC; ++b)
                    if (b < nb) o[b * n] = acc[b];
            }
            __syncthreads();   // stage st is refilled by the next iteration's gather
        }
        return;
    }
    // dense window: pieces of kTB nodes, one chunk of right-hand sides at a time
    for (int bc = 0; bc < nchunks; ++bc) {
#pragma unroll
        for (int b = 0; b < BC; ++b) acc[b] = make_float2(0.f, 0.f);
        for (int c0 = t0; c0 < t1; c0 += kTB) {
            const int cnt = min(kTB, t1 - c0);
            __syncthreads();
            const int p = tile_tabulate(sm, c0, cnt, w, two_over_w, beta, eperm, ecell, efrac, wt);
            tile_gather<BC>(sm, bc, 0, p, src, src_bs, batch);
            cp_async_wait<0>();
            tile_weight<BC>(sm, 0, p);
            __syncthreads();
            tile_accumulate<BC>(sm, acc, 0, c0, max(lo, c0), min(hi, c0 + cnt), g, w);
        }
        if (g < n) {
            const int nb = (int)min((int64_t)BC, batch - (int64_t)bc * BC);
            float2* o = out + (int64_t)bc * BC * n;
#pragma unroll
            for (int b = 0; b < BC; ++b)
                if (b < nb) o[b * n] = acc[b];
        }
    }
}

inline size_t spread_tile_smem(int w, int BC) {
    return 2 * (size_t)BC * kTB * sizeof(float2) + (size_t)kTB * sizeof(float2) + (size_t)kTB * w * sizeof(float) +
           (size_t)kTB * sizeof(int) + (size_t)kTileList * kTB * sizeof(float);
}

// ---- float32 interpolation for many right-hand sides (tiled, pipelined) ---
// One CTA per tile of kInterpNodes sorted slots, all right-hand sides, two
// threads per node (each sums half of a chunk's right-hand sides).  Each
// thread forms the w kernel values of its node once.  The tile's nodes read
// the grid window [cell_first + 1 - w/2, cell_last + w/2] (periodic); for a
// chunk of BC right-hand sides that window is copied into a two-stage ring
// by cp.async while the previous chunk is summed, then every node sums its w
// taps from shared memory and writes dst[b][perm] = sum x wt.  Windows
// longer than kInterpWin points (tiles spanning a sparse stretch of nodes)
// are read from global memory directly.
constexpr int kInterpNodes = 128;
constexpr int kInterpTB = 2 * kInterpNodes;
constexpr int kInterpWin = 384;   // window points per right-hand side
constexpr int kInterpRow = kInterpWin + 4;   // (+4: pair alignment and the pair read past a node's last tap)

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}

// the window of right-hand sides [bc BC, bc BC + BC) into ring stage st: pairs
// (grid indices wsa + 2k, +1, modulo n: n even, so a pair never straddles the
// wrap) or single points (ws + k mod n)
template <int BC>
__device__ __forceinline__ void gather_window(float2* ring, int bc, int st, bool pairs, int npair, int Li, int64_t wsa,
                                              int64_t ws, int64_t n, const float2* __restrict__ grid, int64_t batch) {
    float2* d = ring + st * BC * kInterpRow;
    const int64_t b0 = (int64_t)bc * BC;
    const int nb = (int)min((int64_t)BC, batch - b0);
    const float2* gb = grid + b0 * n;
    if (pairs) {
        for (int k = threadIdx.x; k < npair; k += kInterpTB) {
            int64_t gi = wsa + 2 * k;
            if (gi >= n) gi -= n;
#pragma unroll
            for (int b = 0; b < BC; ++b)
                if (b < nb) cp_async16(&d[b * kInterpRow + 2 * k], gb + b * n + gi);
        }
    } else {
        for (int k = threadIdx.x; k < Li; k += kInterpTB) {
            int64_t gi = ws + k;
            if (gi >= n) gi -= n;
#pragma unroll
            for (int b = 0; b < BC; ++b)
                if (b < nb) cp_async8(&d[b * kInterpRow + k], gb + b * n + gi);
        }
    }
    cp_async_commit();
}

template <int BC>
__global__ void __launch_bounds__(kInterpTB, 4) k_interp_tile(int64_t N, int64_t n, int w, float two_over_w,
                                                           float beta, const int* __restrict__ sperm,
                                                           const int* __restrict__ scell,
                                                           const float* __restrict__ sfrac,
                                                           const float2* __restrict__ grid,
                                                           const float2* __restrict__ wt, float2* __restrict__ dst,
                                                           int64_t dst_bs, int64_t batch) {
    pdl_wait();
    pdl_trigger();
    constexpr int HB = BC / 2;   // right-hand sides per thread and chunk
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* ring = reinterpret_cast<float2*>(smem_raw);   // [2][BC][kInterpRow]
    const int node = threadIdx.x % kInterpNodes, half = threadIdx.x / kInterpNodes;
    const int64_t i0 = (int64_t)blockIdx.x * kInterpNodes;
    const int64_t i = i0 + node;
    const int64_t ilast = min(i0 + (int64_t)kInterpNodes, N) - 1;
    const int h = w / 2;
    const int64_t wa = (int64_t)scell[i0] + 1 - h;            // window start (may be < 0: periodic)
    const int64_t L = (int64_t)scell[ilast] + h - wa + 1;     // window length
    const bool live = i < N;
    // kernel values by tap, shifted by `par` positions: ker[k] = phi(k - par + 1 - h - frac)
    // for 0 <= k - par < w, else 0
    float ker[18];
    int base = 0;
    int c = 0;
    float f = 0.f;
    if (live) {
        c = scell[i];
        f = sfrac[i];
        base = (int)(c + 1 - h - wa);
    }
    auto kernel_values = [&](int par) {
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const int m = k - par;
            ker[k] = (live && m >= 0 && m < w) ? es_kernel<float>((float)(m + 1 - h) - f, two_over_w, beta) : 0.f;
        }
    };
    const int p = live ? sperm[i] : 0;
    const float2 wv = live ? wt[i] : make_float2(0.f, 0.f);
    const int nchunks = (int)((batch + BC - 1) / BC);
    float2 acc[HB];
    if (L <= kInterpWin) {
        int64_t ws = wa % n;
        if (ws < 0) ws += n;
        const bool pairs = (n & 1) == 0;
        const int s0 = pairs ? (int)(ws & 1) : 0;
        const int64_t wsa = ws - s0;
        // (one pair more than the window needs: a node whose taps start at an
        // odd ring index reads w/2 + 1 pairs, the last one past its taps)
        const int npair = (int)((L + s0 + 1) / 2) + 1;
        const int Li = (int)L;
        // with pairs, the kernel values by position in the pairs read from
        // (s0 + base) / 2 on: shifted by the parity of the first tap's ring index
        kernel_values(pairs ? ((s0 + base) & 1) : 0);
        gather_window<BC>(ring, 0, 0, pairs, npair, Li, wsa, ws, n, grid, batch);
        for (int bc = 0; bc < nchunks; ++bc) {
            const int st = bc & 1;
            if (bc + 1 < nchunks) {
                gather_window<BC>(ring, bc + 1, st ^ 1, pairs, npair, Li, wsa, ws, n, grid, batch);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < HB; ++b) acc[b] = make_float2(0.f, 0.f);
            if (pairs) {
                // 16-byte reads of whole pairs: nodes about two grid points
                // apart read consecutive pairs (no bank conflicts); kp holds the
                // kernel values shifted by the parity of the first tap
                const float4* win4 = reinterpret_cast<const float4*>(ring + st * BC * kInterpRow +
                                                                     half * HB * kInterpRow) + (s0 + base) / 2;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    if (q <= w / 2) {
#pragma unroll
                        for (int b = 0; b < HB; ++b) {
                            const float4 v = win4[b * (kInterpRow / 2) + q];
                            // taps in order (the same sums as the per-node kernel
                            // for few right-hand sides; zero weights add exact zeros)
                            acc[b].x = fmaf(ker[2 * q + 1], v.z, fmaf(ker[2 * q], v.x, acc[b].x));
                            acc[b].y = fmaf(ker[2 * q + 1], v.w, fmaf(ker[2 * q], v.y, acc[b].y));
                        }
                    }
                }
            } else {
                const float2* win = ring + st * BC * kInterpRow + half * HB * kInterpRow + s0 + base;
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    if (m < w) {
#pragma unroll
                        for (int b = 0; b < HB; ++b) {
                            const float2 v = win[b * kInterpRow + m];
                            acc[b].x = fmaf(ker[m], v.x, acc[b].x);
                            acc[b].y = fmaf(ker[m], v.y, acc[b].y);
                        }
                    }
                }
            }
            if (live) {
                const int64_t b0 = (int64_t)bc * BC + half * HB;
                float2* o = dst + b0 * dst_bs + p;
#pragma unroll
                for (int b = 0; b < HB; ++b)
                    if (b0 + b < batch) o[b * dst_bs] = cmul(acc[b], wv);
            }
            __syncthreads();   // stage st is refilled by the next iteration's gather
        }
        return;
    }
    // long window: direct gathers
    if (!live) return;
    kernel_values(0);
    int64_t g_first = (int64_t)c + 1 - h;
    if (g_first < 0) g_first += n;
    for (int bc = 0; bc < nchunks; ++bc) {
        const int64_t b0 = (int64_t)bc * BC + half * HB;
#pragma unroll
        for (int b = 0; b < HB; ++b) acc[b] = make_float2(0.f, 0.f);
        int64_t gi = g_first;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            if (m < w) {
#pragma unroll
                for (int b = 0; b < HB; ++b) {
                    if (b0 + b < batch) {
                        const float2 v = grid[(b0 + b) * n + gi];
                        acc[b].x = fmaf(ker[m], v.x, acc[b].x);
                        acc[b].y = fmaf(ker[m], v.y, acc[b].y);
                    }
                }
                if (++gi == n) gi = 0;
            }
        }
#pragma unroll
        for (int b = 0; b < HB; ++b)
            if (b0 + b < batch) dst[(b0 + b) * dst_bs + p] = cmul(acc[b], wv);
    }
}

inline size_t interp_tile_smem(int BC) { return 2 * (size_t)BC * kInterpRow * sizeof(float2); }


__constant__ float2 c_exp2_64[64] = NUFFT_EXP2_64_TABLE;

// The float64 spread with the kernel values and the accumulation in
// double-float arithmetic (float pairs, ~2^-47): on GB300 the float64 pipe
// issues at 1/64 of the float32 rate, and exp/sqrt per tap made the float64
// spread bound by it.  Same gather and tables as k_spread; the float64 inputs
// are converted once per staged node, the outputs once per grid point.
// DDIO (the plan's log-kernel type-1): the strengths come per extended slot,
// already weighted and in double-float (sx[b sx_bs + slot], complex
// double-float), the grid is written in double-float, and every kernel value
// is also stored, in double-float, at ktab[s w + m] (s the node's sorted slot,
// m its tap: grid point cell + 1 - w/2 + m; pre_at points at the count of
// prepended halo slots) for the plan's interpolation on the same geometry and
// kernel, so no value crosses the float64 pipe.
template <int BC, bool DDIO>
__global__ void __launch_bounds__(kTB) k_spread_dd(int64_t n, int w, dd beta,
                                                   const int* __restrict__ cstart, const int* __restrict__ eperm,
                                                   const int* __restrict__ ecell, const double* __restrict__ efrac,
                                                   const double2* __restrict__ src, int64_t src_bs,
                                                   const double2* __restrict__ wt, double2* __restrict__ grid,
                                                   int64_t batch, double* __restrict__ ktab,
                                                   const int* __restrict__ pre_at, int64_t N,
                                                   const cdd* __restrict__ sx, int64_t sx_bs) {
    pdl_wait();
    pdl_trigger();
    __shared__ int s_cell[kChunk];
    __shared__ dd s_frac[kChunk];
    __shared__ cdd s_str[BC][kChunk];
    __shared__ float2 s_exp[64];
    if (threadIdx.x < 64) s_exp[threadIdx.x] = c_exp2_64[threadIdx.x];
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t g = g0 + threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.y * BC;
    const int64_t glast = min(g0 + (int64_t)blockDim.x, n) - 1;
    const int t0 = cstart[g0], t1 = cstart[glast + w];
    int lo = 0, hi = 0;
    if (g < n) { lo = cstart[g]; hi = cstart[g + w]; }
    cdd acc[BC];
#pragma unroll
    for (int b = 0; b < BC; ++b) { acc[b].x = dd(0.f, 0.f); acc[b].y = dd(0.f, 0.f); }
    for (int ch = t0; ch < t1; ch += kChunk) {
        const int cnt = min(kChunk, t1 - ch);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = ch + e;
            s_cell[e] = ecell[i];
            s_frac[e] = dd_from_double(efrac[i]);
            if constexpr (DDIO) {
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    cdd c;
                    c.x = dd(0.f, 0.f);
                    c.y = dd(0.f, 0.f);
                    if (b0 + b < batch) c = sx[(b0 + b) * sx_bs + i];
                    s_str[b][e] = c;
                }
            } else {
                const double2 wv = wt[i];
                const int p = src ? eperm[i] : 0;
#pragma unroll
                for (int b = 0; b < BC; ++b) {
                    double2 v = wv;
                    if (src) v = (b0 + b < batch) ? cmul(src[(b0 + b) * src_bs + p], wv) : make_double2(0.0, 0.0);
                    cdd c;
                    c.x = dd_from_double(v.x);
                    c.y = dd_from_double(v.y);
                    s_str[b][e] = c;
                }
            }
        }
        __syncthreads();
        const int a = max(lo, ch), z = min(hi, ch + cnt);
        const bool keep = DDIO && blockIdx.y == 0;
        const int pre = keep ? *pre_at : 0;
        for (int i = a; i < z; ++i) {
            const int e = i - ch;
            const dd d = dd((float)(int)(g - s_cell[e]), 0.f) - s_frac[e];
            const dd ph = es_kernel_dd(d, 0.5f * (float)w, beta, s_exp);
            if (keep) {
                const int64_t slot = i < pre ? N - pre + i : (i < pre + N ? i - pre : i - pre - N);
                reinterpret_cast<dd*>(ktab)[slot * w + (g - s_cell[e]) + w / 2 - 1] = ph;
            }
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                acc[b].x += ph * s_str[b][e].x;
                acc[b].y += ph * s_str[b][e].y;
            }
        }
    }
    if (g < n) {
#pragma unroll
        for (int b = 0; b < BC; ++b) {
            if (b0 + b < batch) {
                if constexpr (DDIO) reinterpret_cast<cdd*>(grid)[(b0 + b) * n + g] = acc[b];
                else grid[(b0 + b) * n + g] = make_double2(dd_to_double(acc[b].x), dd_to_double(acc[b].y));
            }
        }
    }
}

// The all-float64 path's type-2 interpolation in double-float: the grid comes
// in complex double-float (the FFT leaves it so), the kernel values are formed
// in double-float per node (as in k_interp's float64 case) and the taps are
// summed in double-float on the float32 pipes; one conversion per output, then
// the float64 weight (wt, by sorted slot) and the store at dst[b dst_bs + perm[i]].
template <int BC>
__global__ void __launch_bounds__(kTB) k_interp_dd(int64_t N, int64_t n, int w, dd beta,
                                                   const int* __restrict__ sperm, const int* __restrict__ scell,
                                                   const double* __restrict__ sfrac, const cdd* __restrict__ grid,
                                                   const double2* __restrict__ wt, double2* __restrict__ dst,
                                                   int64_t dst_bs, int64_t batch) {
    pdl_wait();
    pdl_trigger();
    __shared__ float2 s_exp[64];
    if (threadIdx.x < 64) s_exp[threadIdx.x] = c_exp2_64[threadIdx.x];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t b0 = (int64_t)blockIdx.y * BC;
    const int h = w / 2;
    const dd fr = dd_from_double(sfrac[i]);
    dd ker[16];
#pragma unroll
    for (int m = 0; m < 16; ++m)
        ker[m] = (m < w) ? es_kernel_dd(dd((float)(m + 1 - h), 0.f) - fr, 0.5f * (float)w, beta, s_exp) : dd(0.f, 0.f);
    cdd acc[BC];
#pragma unroll
    for (int b = 0; b < BC; ++b) { acc[b].x = dd(0.f, 0.f); acc[b].y = dd(0.f, 0.f); }
    int64_t gi = scell[i] + 1 - h;
    if (gi < 0) gi += n;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (m < w) {
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                if (b0 + b < batch) {
                    const cdd v = grid[(b0 + b) * n + gi];
                    acc[b].x += ker[m] * v.x;
                    acc[b].y += ker[m] * v.y;
                }
            }
            if (++gi == n) gi = 0;
        }
    }
    const int p = sperm[i];
    const double2 wv = wt[i];
#pragma unroll
    for (int b = 0; b < BC; ++b)
        if (b0 + b < batch)
            dst[(b0 + b) * dst_bs + p] = cmul(make_double2(dd_to_double(acc[b].x), dd_to_double(acc[b].y)), wv);
}

// The plan's type-2 for L'(z_p) in double-float: the grid (complex
// double-float) and the kernel values the plan's spread stored (double-float,
// by sorted slot and tap) are combined on the float32 pipes; the sum is
// converted once per node and multiplied by wt (float64, by sorted slot) into
// dst[perm[i]].
__global__ void __launch_bounds__(kTB) k_interp_plan_dd(int64_t N, int64_t n, int w, const int* __restrict__ sperm,
                                                        const int* __restrict__ scell, const cdd* __restrict__ grid,
                                                        const dd* __restrict__ ktab, const double2* __restrict__ wt,
                                                        double2* __restrict__ dst) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int h = w / 2;
    int64_t gi = scell[i] + 1 - h;
    if (gi < 0) gi += n;
    cdd acc;
    acc.x = dd(0.f, 0.f);
    acc.y = dd(0.f, 0.f);
    for (int m = 0; m < w; ++m) {
        const dd k = ktab[i * w + m];
        const cdd v = grid[gi];
        acc.x += k * v.x;
        acc.y += k * v.y;
        if (++gi == n) gi = 0;
    }
    const double2 a = make_double2(dd_to_double(acc.x), dd_to_double(acc.y));
    dst[sperm[i]] = cmul(a, wt[i]);
}

template <typename T, int BC>
__global__ void __launch_bounds__(kTB) k_interp(int64_t N, int64_t n, int w, T two_over_w, T beta,
                                                const int* __restrict__ sperm, const int* __restrict__ scell,
                                                const T* __restrict__ sfrac, const c2<T>* __restrict__ grid,
                                                const c2<T>* __restrict__ wt, c2<T>* __restrict__ dst, int64_t dst_bs,
                                                int64_t batch) {
    pdl_wait();
    pdl_trigger();
    __shared__ float2 s_exp[64];   // float64 data: double-float exponential table
    if constexpr (sizeof(T) == 8) {
        if (threadIdx.x < 64) s_exp[threadIdx.x] = c_exp2_64[threadIdx.x];
        __syncthreads();
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t b0 = (int64_t)blockIdx.y * BC;
    const int c = scell[i];
    const T f = sfrac[i];
    const int h = w / 2;
    T ker[16];
    if constexpr (sizeof(T) == 8) {
        // kernel values in double-float on the float32 pipes (see k_spread_dd)
        const dd fr = dd_from_double((double)f);
        const dd beta_dd((double)beta);
#pragma unroll
        for (int m = 0; m < 16; ++m)
            ker[m] = (m < w) ? (T)dd_to_double(es_kernel_dd(dd((float)(m + 1 - h), 0.f) - fr, 0.5f * (float)w,
                                                            beta_dd, s_exp))
                             : (T)0;
    } else {
#pragma unroll
        for (int m = 0; m < 16; ++m) ker[m] = (m < w) ? es_kernel<T>((T)(m + 1 - h) - f, two_over_w, beta) : (T)0;
    }
    c2<T> acc[BC];
#pragma unroll
    for (int b = 0; b < BC; ++b) acc[b] = mk<T>(0, 0);
    int64_t gi = c + 1 - h;
    if (gi < 0) gi += n;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (m < w) {
#pragma unroll
            for (int b = 0; b < BC; ++b) {
                if (b0 + b < batch) {
                    const c2<T> v = grid[(b0 + b) * n + gi];
                    acc[b].x = fma(ker[m], v.x, acc[b].x);
                    acc[b].y = fma(ker[m], v.y, acc[b].y);
                }
            }
            if (++gi == n) gi = 0;
        }
    }
    const int p = sperm[i];
    const c2<T> wv = wt[i];
#pragma unroll
    for (int b = 0; b < BC; ++b)
        if (b0 + b < batch) dst[(b0 + b) * dst_bs + p] = cmul(acc[b], wv);
}

template <typename T>
__global__ void k_select(const c2<T>* __restrict__ in, int64_t n, c2<T>* __restrict__ out, int64_t out_bs, int64_t P,
                         int64_t K0, const T* __restrict__ fac, int64_t batch) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * batch) return;
    const int64_t b = i / P, k = i - b * P;
    const int64_t src = imod(k - K0, n);
    out[b * out_bs + k] = cscale(in[b * n + src], fac[k]);
}

template <typename T>
__global__ void k_place(const c2<T>* __restrict__ in, int64_t in_bs, int64_t P, int64_t K0, const T* __restrict__ fac,
                        c2<T>* __restrict__ out, int64_t n, int64_t batch, int deriv) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * batch) return;
    const int64_t b = i / n, gidx = i - b * n;
    // centred index of grid slot gidx: k' in [-K0, P - K0)
    const int64_t kc = gidx < n - K0 ? gidx : gidx - n;
    const int64_t k = kc + K0;
    c2<T> v = mk<T>(0, 0);
    if (k >= 0 && k < P) {
        v = cscale(in[b * in_bs + k], fac[k]);
        // derivative coefficients: times j 2 pi k (d/dt of e^{j 2 pi k t})
        if (deriv) v = cscale(cmulj(v, 1), (T)(6.283185307179586476925286766559 * (double)k));
    }
    out[i] = v;
}

template <typename T>
__global__ void k_pointwise(const c2<T>* __restrict__ in, int64_t in_bs, c2<T>* __restrict__ out, int64_t out_bs,
                            int64_t P, const c2<T>* __restrict__ mulc, const T* __restrict__ fac, int64_t batch) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * batch) return;
    const int64_t b = i / P, k = i - b * P;
    c2<T> v = in[b * in_bs + k];
    if (mulc) v = cmul(v, mulc[k]);
    if (fac) v = cscale(v, fac[k]);
    out[b * out_bs + k] = v;
}

// middle stage in linear-convolution form: S_m = c_m + rho^P c_{m+P}, m < P,
// from the length-n (n >= 2P) convolution c of each right-hand side
template <typename T>
__global__ void k_conv_fold(const c2<T>* __restrict__ c, int64_t n, int64_t P, T rhoP, c2<T>* __restrict__ out,
                            int64_t out_bs, int64_t batch) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P * batch) return;
    const int64_t b = i / P, m = i - b * P;
    const c2<T> lo = c[b * n + m], hi = c[b * n + m + P];
    out[b * out_bs + m] = mk<T>(lo.x + rhoP * hi.x, lo.y + rhoP * hi.y);
}

// refinement helpers: widen to float64; r = in - y (in float64, stored in T); out += c
template <typename T>
__global__ void k_widen(const c2<T>* __restrict__ in, double2* __restrict__ out, int64_t n) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { const c2<T> v = in[i]; out[i] = make_double2((double)v.x, (double)v.y); }
}
template <typename T>
__global__ void k_residual(const c2<T>* __restrict__ in, const double2* __restrict__ y, c2<T>* __restrict__ r,
                           int64_t n) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const c2<T> v = in[i];
        const double2 w = y[i];
        r[i] = mk<T>((T)((double)v.x - w.x), (T)((double)v.y - w.y));
    }
}
template <typename T>
__global__ void k_accumulate(c2<T>* __restrict__ out, const c2<T>* __restrict__ c, int64_t n) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = cadd(out[i], c[i]);
}

// node gradient: out[q] = scale * sum_b Re(conj(X[b][q]) Y[b][q]), accumulated in float64
template <typename T>
__global__ void k_grad_nodes(const c2<T>* __restrict__ X, const c2<T>* __restrict__ Y, int64_t N, int64_t batch,
                             double scale, double* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    double acc = 0.0;
    for (int64_t b = 0; b < batch; ++b) {
        const c2<T> x = X[b * N + q], y = Y[b * N + q];
        acc += (double)x.x * (double)y.x + (double)x.y * (double)y.y;
    }
    out[q] = scale * acc;
}

}  // namespace

template <typename T>
void launch_widen(const c2<T>* in, double2* out, int64_t n, cudaStream_t s) {
    Launch L(s, K_POINTWISE, n * (sizeof(c2<T>) + 16.0), sizeof(T) == 8);
    launch_k(k_widen<T>, nblk(n), kTB, 0, s, in, out, n);
}
template <typename T>
void launch_residual(const c2<T>* in, const double2* y, c2<T>* r, int64_t n, cudaStream_t s) {
    Launch L(s, K_POINTWISE, n * (2.0 * sizeof(c2<T>) + 16.0), sizeof(T) == 8);
    launch_k(k_residual<T>, nblk(n), kTB, 0, s, in, y, r, n);
}
template <typename T>
void launch_accumulate(c2<T>* out, const c2<T>* c, int64_t n, cudaStream_t s) {
    Launch L(s, K_POINTWISE, n * 3.0 * sizeof(c2<T>), sizeof(T) == 8);
    launch_k(k_accumulate<T>, nblk(n), kTB, 0, s, out, c, n);
}
#define INST_R(T)                                                                         \
    template void launch_widen<T>(const c2<T>*, double2*, int64_t, cudaStream_t);         \
    template void launch_residual<T>(const c2<T>*, const double2*, c2<T>*, int64_t, cudaStream_t); \
    template void launch_accumulate<T>(c2<T>*, const c2<T>*, int64_t, cudaStream_t);
INST_R(float)
INST_R(double)
#undef INST_R

template <typename T>
void launch_grad_nodes(const c2<T>* X, const c2<T>* Y, int64_t N, int64_t batch, double scale, double* out,
                       cudaStream_t s) {
    Launch L(s, K_POINTWISE, 2.0 * batch * N * sizeof(c2<T>) + 8.0 * N, sizeof(T) == 8);
    launch_k(k_grad_nodes<T>, nblk(N), kTB, 0, s, X, Y, N, batch, scale, out);
}
template void launch_grad_nodes<float>(const float2*, const float2*, int64_t, int64_t, double, double*, cudaStream_t);
template void launch_grad_nodes<double>(const double2*, const double2*, int64_t, int64_t, double, double*,
                                        cudaStream_t);

int64_t geometry_scratch_ints(int64_t N, int64_t n) {
    // cell[N] (+N pad) + frac[N] doubles + count[n+2] + start[n+2] + sums and
    // total (even count) + per-block turn sums (unsigned 64-bit)
    const int64_t nb = (n + 1 + kScanPer - 1) / kScanPer;
    return 4 * N + 2 * (n + 2) + ((nb + 3) & ~(int64_t)1) + 2 * (int64_t)nblk(N);
}

nufft_status build_geometry(Geometry& g, const double* x, uint64_t* T, int64_t N, int64_t n, int w,
                            bool want_float, int* scratch, unsigned long long* sumT, cudaStream_t s) {
    if (n < 2 * w) return fail(NUFFT_ERR_ARG, "grid %lld too small for width %d", (long long)n, w);
    g.N = N; g.n = n; g.w = w;
    int* cell = scratch;
    double* frac = reinterpret_cast<double*>(scratch + 2 * N);   // 8-byte aligned: 2N ints
    int* count = scratch + 4 * N;
    int* start = count + (n + 2);
    g.cell_start = start;
    int* sums = start + (n + 2);
    const int64_t nb = (n + 1 + kScanPer - 1) / kScanPer;
    // 8-byte aligned: every earlier block has an even number of ints
    unsigned long long* partial = reinterpret_cast<unsigned long long*>(sums + ((nb + 3) & ~(int64_t)1));
    const unsigned np = nblk(N);
    NUFFT_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * (n + 1), s));
    { Launch L(s, K_GEOMETRY, 36.0 * N);
      launch_k(k_node_prep, np, kTB, 0, s, x, N, (uint64_t)n, T, cell, frac, count, partial, g.dup_flag); }
    { Launch L(s, K_GEOMETRY, 12.0 * n); launch_k(k_scan_blocks, (unsigned)nb, kScanTB, 0, s, count, n + 1, start, sums); }
    { Launch L(s, K_GEOMETRY, 8.0 * n + 8.0 * np);
      launch_k(k_scan_add, nblk(n + 1), kTB, 0, s, start, n + 1, (const int*)sums, (const unsigned long long*)partial,
               (int64_t)np, sumT); }
    { Launch L(s, K_GEOMETRY, 16.0 * N); launch_k(k_scatter, nblk(N), kTB, 0, s, cell, N, start, count, g.srt_perm); }
    { Launch L(s, K_GEOMETRY, 4.0 * n + 16.0 * N); launch_k(k_order_cells, nblk(n), kTB, 0, s, start, n, T, g.srt_perm); }
    { Launch L(s, K_GEOMETRY, 44.0 * N + 40.0 * N + 8.0 * n);
      launch_k(k_fill, nblk(3 * N + n + w + 1), kTB, 0, s, start, n, w, N, g.srt_perm, cell, frac, T, g.srt_cell,
               g.srt_frac, want_float ? g.srt_fracf : nullptr, g.dup_flag, g.ext_perm, g.ext_cell, g.ext_frac,
               want_float ? g.ext_fracf : nullptr, g.cstart); }
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

template <typename T>
void launch_spread(const Geometry& g, KernelShape ks, const c2<T>* src, int64_t src_bs, const c2<T>* wt_ext,
                   c2<T>* grid, int64_t batch, cudaStream_t s) {
    const T tow = (T)(2.0 / ks.w), beta = (T)ks.beta;
    const T* ef = FracPtr<T>::ext(g);
    // the extended list may carry a wider halo (g.w >= ks.w): cell starts are
    // indexed by cell + g.w/2, so shift them to cell + ks.w/2
    const int* cs = g.cstart + (g.w - ks.w) / 2;
    const double es = sizeof(c2<T>);
    Launch L(s, K_SPREAD, (src ? batch * g.N * es : 0.0) + g.N * (es + 8.0 + sizeof(T)) + 4.0 * (g.n + g.w) +
                              batch * g.n * es, sizeof(T) == 8);
    if constexpr (sizeof(T) == 8) {
        const dd beta_dd(ks.beta);
        const double* efd = g.ext_frac;
        const double2* sd = reinterpret_cast<const double2*>(src);
        const double2* wd = reinterpret_cast<const double2*>(wt_ext);
        double2* gd = reinterpret_cast<double2*>(grid);
        if (batch == 1) {
            launch_k(k_spread_dd<1, false>, dim3(nblk(g.n), 1), kTB, 0, s, g.n, ks.w, beta_dd, cs, g.ext_perm,
                     g.ext_cell, efd, sd, src_bs, wd, gd, batch, (double*)nullptr, g.cstart + g.w / 2, g.N, (const cdd*)nullptr,
                     (int64_t)0);
        } else {
            launch_k(k_spread_dd<4, false>, dim3(nblk(g.n), (unsigned)((batch + 3) / 4)), kTB, 0, s, g.n, ks.w,
                     beta_dd, cs, g.ext_perm, g.ext_cell, efd, sd, src_bs, wd, gd, batch, (double*)nullptr, g.cstart + g.w / 2,
                     g.N, (const cdd*)nullptr, (int64_t)0);
        }
        return;
    }
    if (batch == 1) {
        dim3 gr(nblk(g.n), 1);
        launch_k(k_spread<T, 1>, gr, kTB, 0, s, g.n, ks.w, tow, beta, cs, g.ext_perm, g.ext_cell, ef, src, src_bs,
                                          wt_ext, grid, batch);
    } else if (batch <= 4 || sizeof(T) == 8) {
        dim3 gr(nblk(g.n), (unsigned)((batch + 3) / 4));
        launch_k(k_spread<T, 4>, gr, kTB, 0, s, g.n, ks.w, tow, beta, cs, g.ext_perm, g.ext_cell, ef, src, src_bs,
                                          wt_ext, grid, batch);
    } else if (batch <= 8) {
        dim3 gr(nblk(g.n), (unsigned)((batch + 7) / 8));
        launch_k(k_spread<T, 8>, gr, kTB, 0, s, g.n, ks.w, tow, beta, cs, g.ext_perm, g.ext_cell, ef, src, src_bs,
                                          wt_ext, grid, batch);
    } else if (src) {
        // one CTA per tile of grid points for every right-hand side: the
        // kernel values are formed once per tile and the sample gathers of
        // the next chunk of right-hand sides overlap this chunk's sums
        constexpr int BC = 8;
        const size_t sm = spread_tile_smem(ks.w, BC);
        cudaFuncSetAttribute(k_spread_tile<BC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        launch_k(k_spread_tile<BC>, dim3(nblk(g.n)), kTB, sm, s, g.n, ks.w, (float)tow, (float)beta, cs, g.ext_perm,
                 g.ext_cell, (const float*)ef, (const float2*)src, src_bs, (const float2*)wt_ext, (float2*)grid,
                 batch);
    } else {
        // 16 right-hand sides per block row: each kernel value serves twice as many
        dim3 gr(nblk(g.n), (unsigned)((batch + 15) / 16));
        launch_k(k_spread<T, 16>, gr, kTB, 0, s, g.n, ks.w, tow, beta, cs, g.ext_perm, g.ext_cell, ef, src, src_bs,
                                          wt_ext, grid, batch);
    }
}

template <typename T>
void launch_interp(const Geometry& g, KernelShape ks, const c2<T>* grid, const c2<T>* wt_srt, c2<T>* dst,
                   int64_t dst_bs, int64_t batch, cudaStream_t s) {
    const T tow = (T)(2.0 / ks.w), beta = (T)ks.beta;
    const T* sf = FracPtr<T>::srt(g);
    const double es = sizeof(c2<T>);
    Launch L(s, K_INTERP, batch * g.n * es + g.N * (8.0 + sizeof(T) + es) + batch * g.N * es, sizeof(T) == 8);
    if (batch == 1) {
        dim3 gr(nblk(g.N), 1);
        launch_k(k_interp<T, 1>, gr, kTB, 0, s, g.N, g.n, ks.w, tow, beta, g.srt_perm, g.srt_cell, sf, grid, wt_srt, dst,
                                          dst_bs, batch);
    } else if (batch <= 4 || sizeof(T) == 8) {
        dim3 gr(nblk(g.N), (unsigned)((batch + 3) / 4));
        launch_k(k_interp<T, 4>, gr, kTB, 0, s, g.N, g.n, ks.w, tow, beta, g.srt_perm, g.srt_cell, sf, grid, wt_srt, dst,
                                          dst_bs, batch);
    } else {
        // one CTA per tile of sorted nodes for every right-hand side: kernel
        // values once per node, the grid window of the next chunk of
        // right-hand sides copied while this chunk is summed
        constexpr int BC = 8;
        const size_t sm = interp_tile_smem(BC);
        cudaFuncSetAttribute(k_interp_tile<BC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        launch_k(k_interp_tile<BC>, dim3(nblk(g.N, kInterpNodes)), kInterpTB, sm, s, g.N, g.n, ks.w, (float)tow,
                 (float)beta, g.srt_perm, g.srt_cell, (const float*)sf, (const float2*)grid, (const float2*)wt_srt,
                 (float2*)dst, dst_bs, batch);
    }
}

void launch_spread_plan_dd(const Geometry& g, KernelShape ks, const void* sx, int64_t sx_bs, void* grid,
                           int64_t batch, cudaStream_t s, void* ktab) {
    const int* cs = g.cstart + (g.w - ks.w) / 2;
    Launch L(s, K_SPREAD, batch * 2.0 * g.N * 16.0 + g.N * (8.0 + 8.0) + 4.0 * (g.n + g.w) + batch * g.n * 16.0 +
                              g.N * ks.w * 8.0, true);
    const dd beta_dd(ks.beta);
    launch_k(k_spread_dd<4, true>, dim3(nblk(g.n), (unsigned)((batch + 3) / 4)), kTB, 0, s, g.n, ks.w, beta_dd, cs,
             g.ext_perm, g.ext_cell, (const double*)g.ext_frac, (const double2*)nullptr, (int64_t)0,
             (const double2*)nullptr, static_cast<double2*>(grid), batch, static_cast<double*>(ktab),
             g.cstart + g.w / 2, g.N, static_cast<const cdd*>(sx), sx_bs);
}

void launch_interp_dd(const Geometry& g, KernelShape ks, const void* grid, const double2* wt_srt, double2* dst,
                      int64_t dst_bs, int64_t batch, cudaStream_t s) {
    Launch L(s, K_INTERP, batch * g.n * 16.0 + g.N * (8.0 + 8.0 + 16.0) + batch * g.N * 16.0, true);
    const dd beta_dd(ks.beta);
    const cdd* gd = static_cast<const cdd*>(grid);
    if (batch <= 2) {
        launch_k(k_interp_dd<2>, dim3(nblk(g.N), (unsigned)((batch + 1) / 2)), kTB, 0, s, g.N, g.n, ks.w, beta_dd,
                 g.srt_perm, g.srt_cell, (const double*)g.srt_frac, gd, wt_srt, dst, dst_bs, batch);
    } else {
        launch_k(k_interp_dd<8>, dim3(nblk(g.N), (unsigned)((batch + 7) / 8)), kTB, 0, s, g.N, g.n, ks.w, beta_dd,
                 g.srt_perm, g.srt_cell, (const double*)g.srt_frac, gd, wt_srt, dst, dst_bs, batch);
    }
}

void launch_interp_plan_dd(const Geometry& g, KernelShape ks, const void* grid, const void* ktab, const double2* wt,
                           double2* dst, cudaStream_t s) {
    Launch L(s, K_INTERP, g.N * ks.w * (16.0 + 8.0) + g.N * (8.0 + 16.0 + 16.0), true);
    launch_k(k_interp_plan_dd, nblk(g.N), kTB, 0, s, g.N, g.n, ks.w, g.srt_perm, g.srt_cell,
             static_cast<const cdd*>(grid), static_cast<const dd*>(ktab), wt, dst);
}

template <typename T>
void launch_select(const c2<T>* in, int64_t n, c2<T>* out, int64_t out_bs, int64_t P, int64_t K0, const T* fac,
                   int64_t batch, cudaStream_t s) {
    Launch L(s, K_SELECT, 2.0 * batch * P * sizeof(c2<T>) + P * sizeof(T), sizeof(T) == 8);
    launch_k(k_select<T>, nblk(P * batch), kTB, 0, s, in, n, out, out_bs, P, K0, fac, batch);
}

template <typename T>
void launch_place(const c2<T>* in, int64_t in_bs, int64_t P, int64_t K0, const T* fac, c2<T>* out, int64_t n,
                  int64_t batch, cudaStream_t s, bool deriv) {
    Launch L(s, K_PLACE, batch * (P + n) * sizeof(c2<T>) + P * sizeof(T), sizeof(T) == 8);
    launch_k(k_place<T>, nblk(n * batch), kTB, 0, s, in, in_bs, P, K0, fac, out, n, batch, deriv ? 1 : 0);
}

template <typename T>
void launch_conv_fold(const c2<T>* c, int64_t n, int64_t P, double rhoP, c2<T>* out, int64_t out_bs, int64_t batch,
                      cudaStream_t s) {
    Launch L(s, K_POINTWISE, 3.0 * batch * P * sizeof(c2<T>), sizeof(T) == 8);
    launch_k(k_conv_fold<T>, nblk(P * batch), kTB, 0, s, c, n, P, (T)rhoP, out, out_bs, batch);
}

template <typename T>
void launch_pointwise(const c2<T>* in, int64_t in_bs, c2<T>* out, int64_t out_bs, int64_t P, const c2<T>* mulc,
                      const T* fac, int64_t batch, cudaStream_t s) {
    Launch L(s, K_POINTWISE, 2.0 * batch * P * sizeof(c2<T>) + (mulc ? P * sizeof(c2<T>) : 0) +
                                 (fac ? P * sizeof(T) : 0), sizeof(T) == 8);
    launch_k(k_pointwise<T>, nblk(P * batch), kTB, 0, s, in, in_bs, out, out_bs, P, mulc, fac, batch);
}

#define INST(T)                                                                                                  \
    template void launch_spread<T>(const Geometry&, KernelShape, const c2<T>*, int64_t, const c2<T>*, c2<T>*,   \
                                   int64_t, cudaStream_t);                                                       \
    template void launch_interp<T>(const Geometry&, KernelShape, const c2<T>*, const c2<T>*, c2<T>*, int64_t,   \
                                   int64_t, cudaStream_t);                                                       \
    template void launch_select<T>(const c2<T>*, int64_t, c2<T>*, int64_t, int64_t, int64_t, const T*, int64_t, \
                                   cudaStream_t);                                                                \
    template void launch_place<T>(const c2<T>*, int64_t, int64_t, int64_t, const T*, c2<T>*, int64_t, int64_t,  \
                                  cudaStream_t, bool);                                                           \
    template void launch_conv_fold<T>(const c2<T>*, int64_t, int64_t, double, c2<T>*, int64_t, int64_t,         \
                                      cudaStream_t);                                                             \
    template void launch_pointwise<T>(const c2<T>*, int64_t, c2<T>*, int64_t, int64_t, const c2<T>*, const T*,  \
                                      int64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace nufft45

namespace nufft45 {
namespace {
__global__ void k_debug_dd_exp(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    __shared__ float2 s_exp[64];
    if (threadIdx.x < 64) s_exp[threadIdx.x] = c_exp2_64[threadIdx.x];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = x[i];
        const float hi = (float)v;
        const dd e = dd_exp_nonpos(dd(hi, (float)(v - (double)hi)), s_exp);
        out[i] = (double)e.hi + (double)e.lo;
    }
}
}  // namespace
}  // namespace nufft45

// Test hook (not part of the public header): out[i] = e^{x[i]} by the
// double-float exponential of the plan's spreading kernels (dd_exp_nonpos,
// valid for -87 < x <= 0); device arrays of n float64 values.
extern "C" nufft_status nufft_debug_dd_exp(int64_t n, const double* x, double* out, nufft_stream_t stream) {
    using namespace nufft45;
    if (n < 0 || (n > 0 && (!x || !out))) return fail(NUFFT_ERR_ARG, "bad exp test arguments");
    if (n == 0) return NUFFT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    launch_k(k_debug_dd_exp, nblk(n), kTB, 0, s, x, n, out);
    NUFFT_CUDA_TRY(cudaGetLastError());
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}

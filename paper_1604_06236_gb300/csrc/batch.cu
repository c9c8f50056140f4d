// Batched type-4/5 inverses of many independent instances of uneven size in
// one persistent kernel.
//
// Every CTA takes instances from a work queue (an atomic counter over the
// descriptors, which the host orders by decreasing N) and runs the whole
// method for one instance with all its threads: the float64 plan of Sec. III
// (exact turns, counting sort by cell, the log-kernel type-1 as eta
// type-1s of length N, the fold of Eq. 7, kernel samples (Eq. 29), Lagrange
// coefficients (Eq. 43), L'(z_p) by a type-2 (Eq. 16), weights (Eqs. 27, 40))
// followed by the float32 type-5 (Fig. 1) or type-4 (Fig. 2) inverse.
// Stages are separated by block barriers; arrays live in a per-CTA scratch
// slab.  Every FFT inside is a power of two: grids are rounded up to one, and
// lengths N that are not use Bluestein's chirp-z on a power-of-two length, so
// one table of W_{2^L} twiddles serves all instances.  The plan's
// float64-class arithmetic (its FFTs, spreading and interpolation) runs in
// double-float (pairs of float32, ~2^-48) on the float32 pipes; float64 is
// kept for the per-node phases, exponentials and the weights.
#include "internal.h"
#include "cis64.cuh"
#include "df.cuh"
#include "fft_p2.cuh"

#include <algorithm>
#include <cstring>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace nufft45 {
namespace {

constexpr int kMaxLog = 16;                 // largest power-of-two FFT inside: 2^16
constexpr int kMaxEta = 4;                  // largest log-kernel oversampling (Sec. V)
constexpr int kMaxW = 16;                   // largest spreading width

struct Desc {
    int64_t N;
    const double* x;
    const float2* in;
    float2* out;
    int kind;          // 5 or 4
    int log_ns;        // transforms' grid 2^log_ns >= 2N
    int log_m;         // FFT length for size-N transforms (N itself if a power of two, else Bluestein)
    int pow2;          // N is a power of two
    int64_t tab;       // offset of this grid's deconvolution tables
    int64_t slot;      // index into the status array
};

struct Args {
    const Desc* desc;
    int count;
    int* counter;
    int* status;
    char* scratch;
    size_t scratch_per_cta;
    const cdd* twdd;         // W_{2^kMaxLog}^e in double-float
    const float2* tw32;
    const double* dec_plan;  // 1/phihat (plan width) per grid, centred index
    const float* dec_solve;  // 1/phihat (transforms' width)
    double beta_plan, beta_solve;
    int max_rl;              // largest FFT radix inside: 2^max_rl (2 or 3)
    // the method's parameters (Sec. V): gamma = rho^-N, eta <= kMaxEta, the
    // spreading widths of the float64-class plan and of the float32 transforms
    double gamma;
    int eta, w_plan, w_solve;
};

// ---------------------------------------------------------------- helpers
template <typename X> __device__ __forceinline__ X* carve(char*& p, size_t count) {
    X* r = reinterpret_cast<X*>(p);
    p += (count * sizeof(X) + 255) & ~(size_t)255;
    return r;
}

// 2^(j/64) in double-float for the double-float kernel values
__constant__ float2 c_exp2_64b[64] = NUFFT_EXP2_64_TABLE;

__device__ __forceinline__ cdd to_cdd(double2 v) {
    cdd r;
    r.x = dd_from_double(v.x);
    r.y = dd_from_double(v.y);
    return r;
}

// one radix-R stage of a block-wide Stockham FFT (R a compile-time constant so
// the R values of a butterfly stay in registers)
template <typename T, int R>
__device__ __forceinline__ void cta_fft_stage(const c2<T>* src, c2<T>* dst, int n, int ns_log, int dir,
                                              const c2<T>* __restrict__ tw) {
    constexpr int rl = R == 8 ? 3 : (R == 4 ? 2 : 1);
    const int nr = n >> rl;
    for (int j = threadIdx.x; j < nr; j += blockDim.x) {
        c2<T> v[R];
        const int jm = j & ((1 << ns_log) - 1);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            c2<T> x = src[j + k * nr];
            if (jm && k) {
                // W_{Ns R}^{jm k} = W_{2^kMaxLog}^{jm k 2^(kMaxLog - log(Ns R))}
                c2<T> w = ldg(&tw[(jm * k) << (kMaxLog - ns_log - rl)]);
                if (dir > 0) w.y = -w.y;
                x = cmul(x, w);
            }
            v[k] = x;
        }
        p2::dft_reg<R, T>(v, dir);
        c2<T>* d = dst + ((j >> ns_log) << (ns_log + rl)) + jm;
#pragma unroll
        for (int m = 0; m < R; ++m) d[m << ns_log] = v[m];
    }
}

// block-wide power-of-two Stockham FFT of length 2^logn over global scratch,
// radix 8/4/2 stages; dir -1 forward, +1 inverse, unnormalised.  Returns the
// buffer that holds the result.
template <typename T>
__device__ c2<T>* cta_fft(c2<T>* buf, c2<T>* work, int logn, int dir, const c2<T>* __restrict__ tw, int max_rl) {
    const int n = 1 << logn;
    c2<T>* src = buf;
    c2<T>* dst = work;
    int ns_log = 0;
    while (ns_log < logn) {
        const int rem = logn - ns_log;
        const int rl = rem >= max_rl ? max_rl : rem;
        if (rl == 3) cta_fft_stage<T, 8>(src, dst, n, ns_log, dir, tw);
        else if (rl == 2) cta_fft_stage<T, 4>(src, dst, n, ns_log, dir, tw);
        else cta_fft_stage<T, 2>(src, dst, n, ns_log, dir, tw);
        __syncthreads();
        c2<T>* t = src; src = dst; dst = t;
        ns_log += rl;
    }
    return src;
}

// chirp c_k = e^{+j pi k^2 / N} (k^2 reduced exactly mod 2N)
__device__ __forceinline__ double2 chirp64(int64_t k, int64_t N) {
    const uint64_t e = ((uint64_t)k * (uint64_t)k) % (uint64_t)(2 * N);
    double s, c;
    sincospi((double)e / (double)N, &s, &c);
    return make_double2(c, s);
}

// Bluestein context of one instance: chirps and filter spectra (forward: H,
// inverse: conj(H(-k))), with the 1/M scaling folded in
template <typename T> struct Blue {
    const c2<T>* chirp;   // N
    const c2<T>* H;       // M
    c2<T>* A;             // M
    c2<T>* W;             // M
};

// length-N DFT, dir -1: X_k = sum x_j e^{-j 2 pi jk/N}; +1 with e^{+}.
// In place on x (N values); `w` is N (+) scratch when N is a power of two.
template <typename T>
__device__ void cta_dft(c2<T>* x, c2<T>* w, const Desc& d, int dir, const Blue<T>& bl, const c2<T>* tw, int max_rl) {
    const int64_t N = d.N;
    if (d.pow2) {
        c2<T>* r = cta_fft<T>(x, w, d.log_m, dir, tw, max_rl);
        if (r != x)
            for (int64_t i = threadIdx.x; i < N; i += blockDim.x) x[i] = r[i];
        __syncthreads();
        return;
    }
    const int64_t M = (int64_t)1 << d.log_m;
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        c2<T> v = mk<T>(0, 0);
        if (i < N) v = dir < 0 ? cmulc(x[i], bl.chirp[i]) : cmul(x[i], bl.chirp[i]);
        bl.A[i] = v;
    }
    __syncthreads();
    c2<T>* r = cta_fft<T>(bl.A, bl.W, d.log_m, -1, tw, max_rl);
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        c2<T> h = dir < 0 ? bl.H[i] : cconj(bl.H[i ? M - i : 0]);
        r[i] = cmul(r[i], h);
    }
    __syncthreads();
    c2<T>* r2 = cta_fft<T>(r, r == bl.A ? bl.W : bl.A, d.log_m, +1, tw, max_rl);
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
        x[i] = dir < 0 ? cmulc(r2[i], bl.chirp[i]) : cmul(r2[i], bl.chirp[i]);
    __syncthreads();
}

// block-wide exclusive scan of cnt[0..n) into out[0..n], out[n] = total
__device__ void cta_scan(const int* cnt, int n, int* out, int* s_part) {
    const int nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    const int a = threadIdx.x * per, b = min(n, a + per);
    int sum = 0;
    for (int i = a; i < b; ++i) sum += cnt[i];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < nt; ++t) { const int v = s_part[t]; s_part[t] = acc; acc += v; }
        out[n] = acc;
    }
    __syncthreads();
    int acc = s_part[threadIdx.x];
    for (int i = a; i < b; ++i) { const int v = cnt[i]; out[i] = acc; acc += v; }
    __syncthreads();
}

// ---------------------------------------------------------------- kernel
__global__ void __launch_bounds__(512) k_batch(Args a) {
    __shared__ int s_item;
    __shared__ int s_part[1024];
    __shared__ unsigned long long s_sum[32];
    __shared__ float2 s_exp[64];
    char* const base = a.scratch + (size_t)blockIdx.x * a.scratch_per_cta;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid < 64) s_exp[tid] = c_exp2_64b[tid];
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= a.count) break;
        const Desc d = a.desc[it];
        const int64_t N = d.N;
        const int ns = 1 << d.log_ns;
        const int64_t M = (int64_t)1 << d.log_m;
        const int64_t K0 = N / 2;
        const int eta = a.eta, w_plan = a.w_plan, w_solve = a.w_solve;
        const double log_rho = -log(a.gamma) / (double)N;
        const double rhoN = 1.0 / a.gamma;
        const double* dec_p = a.dec_plan + d.tab;
        const float* dec_s = a.dec_solve + d.tab;
        // ---- scratch layout
        char* p = base;
        uint64_t* T = carve<uint64_t>(p, N);
        int* cell = carve<int>(p, N);
        double* frac = carve<double>(p, N);
        int* perm = carve<int>(p, N);
        int* cnt = carve<int>(p, ns + 1);
        int* start = carve<int>(p, ns + 1);
        double2* modm = carve<double2>(p, N);
        double2* modp = carve<double2>(p, N);
        cdd* str = carve<cdd>(p, (size_t)eta * N);    // log-kernel strengths (double-float)
        cdd* G = carve<cdd>(p, (size_t)eta * ns);
        cdd* GW = carve<cdd>(p, (size_t)ns);
        cdd* v64 = carve<cdd>(p, M);
        cdd* w64v = carve<cdd>(p, M);
        double2* K64 = carve<double2>(p, N);
        double2* D64 = carve<double2>(p, N);
        cdd* chirp_d = carve<cdd>(p, N);
        cdd* H_d = carve<cdd>(p, M);
        cdd* A_d = carve<cdd>(p, M);
        cdd* W_d = carve<cdd>(p, M);
        float2* chirp_f = carve<float2>(p, N);
        float2* H_f = carve<float2>(p, M);
        float2* A_f = carve<float2>(p, M);
        float2* W_f = carve<float2>(p, M);
        float2* K32 = carve<float2>(p, N);
        float2* wm32 = carve<float2>(p, N);   // w e^{-+ j 2 pi K0 t} for the solve
        float2* g32 = carve<float2>(p, ns);
        float2* gw32 = carve<float2>(p, ns);
        float2* vec32 = carve<float2>(p, M);
        float2* vw32 = carve<float2>(p, M);
        dd* fracd = carve<dd>(p, N);
        float* fracf = carve<float>(p, N);
        Blue<dd> bd{chirp_d, H_d, A_d, W_d};
        Blue<float> bf{chirp_f, H_f, A_f, W_f};

        // ---- nodes: exact turns, their sum mod 2^64, cells on the grid
        unsigned long long part = 0;
        for (int64_t i = tid; i < N; i += nt) {
            double u = d.x[i] / 6.283185307179586476925286766559;
            u -= floor(u);
            if (u >= 1.0) u = 0.0;
            const uint64_t t = __double2ull_rz(u * 18446744073709551616.0);
            T[i] = t;
            part += t;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if ((tid & 31) == 0) s_sum[tid >> 5] = part;
        for (int64_t c = tid; c <= ns; c += nt) cnt[c] = 0;
        __syncthreads();
        unsigned long long sumT = 0;
        for (int wv = 0; wv < (nt >> 5); ++wv) sumT += s_sum[wv];
        for (int64_t i = tid; i < N; i += nt) {
            const uint64_t t = T[i];
            const int c = (int)__umul64hi(t, (uint64_t)ns);
            cell[i] = c;
            const double fr = (double)(t * (uint64_t)ns) * 5.42101086242752217003726400434970855712890625e-20;
            frac[i] = fr;
            fracd[i] = dd_from_double(fr);
            fracf[i] = (float)fr;
            atomicAdd(&cnt[c], 1);
            const double2 mm = cis_turns_t((uint64_t)K0 * t, -1);
            modm[i] = mm;
            modp[i] = make_double2(mm.x, -mm.y);
            // strengths e^{-j 2 pi N r t} e^{-j 2 pi K0 t} as powers of
            // beta = e^{-j 2 pi N t}, in double-float
            cdd sv = to_cdd(mm);
            const cdd bt = to_cdd(cis_turns_t((uint64_t)N * t, -1));
            for (int r = 0; r < eta; ++r) {
                str[(int64_t)r * N + i] = sv;
                sv = cmul(sv, bt);
            }
        }
        __syncthreads();
        cta_scan(cnt, ns, start, s_part);
        for (int64_t c = tid; c <= ns; c += nt) cnt[c] = 0;
        __syncthreads();
        for (int64_t i = tid; i < N; i += nt) {
            const int c = cell[i];
            perm[start[c] + atomicAdd(&cnt[c], 1)] = (int)i;
        }
        __syncthreads();
        // order each cell by (T, index); flag coincident neighbours
        for (int64_t c = tid; c < ns; c += nt) {
            const int lo = start[c], hi = start[c + 1];
            for (int i = lo + 1; i < hi; ++i) {
                const int q = perm[i];
                const uint64_t tq = T[q];
                int j = i - 1;
                while (j >= lo && (T[perm[j]] > tq || (T[perm[j]] == tq && perm[j] > q))) { perm[j + 1] = perm[j]; --j; }
                perm[j + 1] = q;
            }
        }
        __syncthreads();
        for (int64_t i = tid; i < N; i += nt) {
            if (N > 1 && T[perm[i + 1 < N ? i + 1 : 0]] - T[perm[i]] < (1ull << 20)) a.status[d.slot] = NUFFT_ERR_DUP_NODES;
        }

        // ---- Bluestein chirps and filter spectra (double-float, float32 copies)
        if (!d.pow2) {
            for (int64_t i = tid; i < M; i += nt) {
                int64_t k = -1;
                if (i < N) k = i; else if (i > M - N) k = M - i;
                cdd c = mk<dd>(0, 0);
                if (k >= 0) {
                    const double2 cv = chirp64(k, N);
                    c = to_cdd(cv);
                    if (i < N) chirp_f[i] = make_float2((float)cv.x, (float)cv.y);
                }
                A_d[i] = c;
                if (i < N) chirp_d[i] = c;
            }
            __syncthreads();
            cdd* h = cta_fft<dd>(A_d, W_d, d.log_m, -1, a.twdd, a.max_rl);
            const float invM = 1.0f / (float)M;   // a power of two: exact
            for (int64_t i = tid; i < M; i += nt) {
                cdd v;
                v.x = dd_mul_f(h[i].x, invM);
                v.y = dd_mul_f(h[i].y, invM);
                H_d[i] = v;
                H_f[i] = make_float2(v.x.hi, v.y.hi);
            }
            __syncthreads();
        }

        // ---- log-kernel spectrum: eta type-1s of length N on the grid
        // (double-float kernel values and sums)
        const float hp = 0.5f * (float)w_plan;
        const dd beta_p(a.beta_plan);
        for (int g = tid; g < ns; g += nt) {
            cdd acc[kMaxEta];
#pragma unroll
            for (int r = 0; r < kMaxEta; ++r) acc[r] = mk<dd>(0, 0);
            for (int j = 0; j < w_plan; ++j) {
                const int cu = g - w_plan / 2 + j;                  // unwrapped cell
                const int cw = cu < 0 ? cu + ns : (cu >= ns ? cu - ns : cu);
                for (int i = start[cw]; i < start[cw + 1]; ++i) {
                    const int q = perm[i];
                    const dd ph = es_kernel_dd(dd((float)(g - cu), 0.f) - fracd[q], hp, beta_p, s_exp);
#pragma unroll
                    for (int r = 0; r < kMaxEta; ++r) {
                        if (r < eta) {
                            const cdd sv = str[(int64_t)r * N + q];
                            acc[r].x += ph * sv.x;
                            acc[r].y += ph * sv.y;
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < kMaxEta; ++r)
                if (r < eta) G[(int64_t)r * ns + g] = acc[r];
        }
        __syncthreads();
        for (int r = 0; r < eta; ++r) {
            cdd* res = cta_fft<dd>(G + (int64_t)r * ns, GW, d.log_ns, -1, a.twdd, a.max_rl);
            if (res != G + (int64_t)r * ns)
                for (int g = tid; g < ns; g += nt) G[(int64_t)r * ns + g] = res[g];
            __syncthreads();
        }
        // fold (Eq. 7) with Lambda_k = -rho^k / k (Eq. 41) and the deconvolution;
        // rho^{N r + m} = gamma^{-r} rho^m
        for (int64_t m = tid; m < N; m += nt) {
            const int64_t kc = m - K0;
            const int64_t src = kc < 0 ? kc + ns : kc;
            const double dec = dec_p[kc + ns / 2];
            const double rm = exp((double)m * log_rho);
            cdd acc = mk<dd>(0, 0);
            double gr = 1.0;
            for (int r = 0; r < eta; ++r, gr *= rhoN) {
                const int64_t k = N * r + m;
                if (k == 0) continue;
                const dd lam = dd_from_double(-gr * rm / (double)k * dec);
                const cdd b = G[(int64_t)r * ns + src];
                acc.x += lam * b.x;
                acc.y += lam * b.y;
            }
            v64[m] = acc;
        }
        __syncthreads();
        cta_dft<dd>(v64, w64v, d, +1, bd, a.twdd, a.max_rl);
        // K_q (Eq. 29), then F = DFT(K) for Eq. 43
        const uint64_t Cph = (uint64_t)sumT + (uint64_t)N * 0x8000000000000000ull;
        for (int64_t q = tid; q < N; q += nt) {
            const cdd vq = v64[q];
            double s, c;
            sincospi(dd_to_double(vq.y) / 3.141592653589793238462643383279502884 + 2.0 * turns_of(Cph), &s, &c);
            const double mag = exp(dd_to_double(vq.x));
            const double2 k = make_double2(mag * c, mag * s);
            K64[q] = k;
            K32[q] = make_float2((float)k.x, (float)k.y);
            v64[q] = to_cdd(k);
        }
        __syncthreads();
        cta_dft<dd>(v64, w64v, d, -1, bd, a.twdd, a.max_rl);
        // d_m = (m+1) L_{m+1}, L_k = F_k rho^-k / N (k >= 1), L_N = 1; placed on
        // the grid with the plan's deconvolution (type-2, Eq. 16)
        for (int g = tid; g < ns; g += nt) {
            const int64_t kc = g < ns - K0 ? g : g - ns;
            const int64_t m = kc + K0;
            cdd v = mk<dd>(0, 0);
            if (m >= 0 && m < N) {
                const int64_t k = m + 1;
                double f = (double)k * dec_p[kc + ns / 2];
                if (k < N) {
                    f *= exp(-(double)k * log_rho) / (double)N;
                    const dd fd = dd_from_double(f);
                    v.x = fd * v64[k].x;
                    v.y = fd * v64[k].y;
                } else {
                    v.x = dd_from_double(f);
                }
            }
            G[g] = v;
        }
        __syncthreads();
        {
            cdd* gsp = cta_fft<dd>(G, GW, d.log_ns, +1, a.twdd, a.max_rl);
            // L'(z_p) by interpolation (double-float); then w_p (Eqs. 27, 40)
            for (int64_t i = tid; i < N; i += nt) {
                const int c = cell[i];
                const dd fdd = fracd[i];
                cdd acc = mk<dd>(0, 0);
                for (int m = 0; m < w_plan; ++m) {
                    int gi = c + 1 - w_plan / 2 + m;
                    gi = gi < 0 ? gi + ns : (gi >= ns ? gi - ns : gi);
                    const dd ph = es_kernel_dd(dd((float)(m + 1 - w_plan / 2), 0.f) - fdd, hp, beta_p, s_exp);
                    const cdd gv = gsp[gi];
                    acc.x += ph * gv.x;
                    acc.y += ph * gv.y;
                }
                const double2 Dp = cmul(make_double2(dd_to_double(acc.x), dd_to_double(acc.y)), modp[i]);
                D64[i] = Dp;
                const uint64_t t = T[i];
                const double2 e = cis_turns_t((uint64_t)N * t, -1);
                const double2 z = cis_turns_t(t, +1);
                const double2 h = make_double2(rhoN * e.x - 1.0, rhoN * e.y);
                const double2 den = cmul(h, cmul(Dp, z));
                const double nn = den.x * den.x + den.y * den.y;
                const double2 w = make_double2(den.x / nn, -den.y / nn);
                const double2 wm = cmul(w, d.kind == 5 ? modm[i] : modp[i]);
                wm32[i] = make_float2((float)wm.x, (float)wm.y);
            }
        }
        __syncthreads();

        // ---- the float32 inverse (its scalings rho^{+-k} in float32: |k log rho|
        // <= log gamma, so expf is accurate to a few float32 ulp)
        const float tow_s = 2.0f / (float)w_solve;
        const float beta_s = (float)a.beta_solve;
        const float lr = (float)log_rho, invN = 1.0f / (float)N;
        if (d.kind == 5) {
            // a_p = s_p w_p e^{-j 2 pi K0 t_p}: type-1 (gather), FFT, deconvolve x rho^k
            for (int g = tid; g < ns; g += nt) {
                float2 acc = make_float2(0.f, 0.f);
                for (int j = 0; j < w_solve; ++j) {
                    const int cu = g - w_solve / 2 + j;
                    const int cw = cu < 0 ? cu + ns : (cu >= ns ? cu - ns : cu);
                    for (int i = start[cw]; i < start[cw + 1]; ++i) {
                        const int q = perm[i];
                        const float ph = es_kernel<float>((float)(g - cu) - fracf[q], tow_s, beta_s);
                        const float2 sv = cmul(d.in[q], wm32[q]);
                        acc.x = fmaf(ph, sv.x, acc.x);
                        acc.y = fmaf(ph, sv.y, acc.y);
                    }
                }
                g32[g] = acc;
            }
            __syncthreads();
            float2* B = cta_fft<float>(g32, gw32, d.log_ns, -1, a.tw32, a.max_rl);
            for (int64_t k = tid; k < N; k += nt) {
                const int64_t kc = k - K0;
                const float f = expf((float)k * lr) * dec_s[kc + ns / 2];
                vec32[k] = cscale(B[kc < 0 ? kc + ns : kc], f);
            }
            __syncthreads();
            cta_dft<float>(vec32, vw32, d, +1, bf, a.tw32, a.max_rl);
            for (int64_t q = tid; q < N; q += nt) vec32[q] = cmul(vec32[q], K32[q]);
            __syncthreads();
            cta_dft<float>(vec32, vw32, d, -1, bf, a.tw32, a.max_rl);
            for (int64_t m = tid; m < N; m += nt)
                d.out[m] = cscale(vec32[m], expf(-(float)m * lr) * invN);
            __syncthreads();
        } else {
            for (int64_t k = tid; k < N; k += nt) vec32[k] = cscale(d.in[k], expf((float)k * lr));
            __syncthreads();
            cta_dft<float>(vec32, vw32, d, +1, bf, a.tw32, a.max_rl);
            for (int64_t q = tid; q < N; q += nt) vec32[q] = cmul(vec32[q], K32[q]);
            __syncthreads();
            cta_dft<float>(vec32, vw32, d, -1, bf, a.tw32, a.max_rl);
            for (int g = tid; g < ns; g += nt) {
                const int64_t kc = g < ns - K0 ? g : g - ns;
                const int64_t m = kc + K0;
                float2 v = make_float2(0.f, 0.f);
                if (m >= 0 && m < N)
                    v = cscale(vec32[m], expf(-(float)m * lr) * invN * dec_s[kc + ns / 2]);
                g32[g] = v;
            }
            __syncthreads();
            float2* gsp = cta_fft<float>(g32, gw32, d.log_ns, +1, a.tw32, a.max_rl);
            for (int64_t i = tid; i < N; i += nt) {
                const int c = cell[i];
                const float f = fracf[i];
                float2 acc = make_float2(0.f, 0.f);
                for (int m = 0; m < w_solve; ++m) {
                    int gi = c + 1 - w_solve / 2 + m;
                    gi = gi < 0 ? gi + ns : (gi >= ns ? gi - ns : gi);
                    const float ph = es_kernel<float>((float)(m + 1 - w_solve / 2) - f, tow_s, beta_s);
                    acc.x = fmaf(ph, gsp[gi].x, acc.x);
                    acc.y = fmaf(ph, gsp[gi].y, acc.y);
                }
                d.out[i] = cmul(acc, wm32[i]);
            }
            __syncthreads();
        }
    }
}

__global__ void k_twiddle_table(int logn, cdd* tdd, float2* t32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (1 << logn)) return;
    double s, c;
    sincospi(-2.0 * (double)i / (double)(1 << logn), &s, &c);
    tdd[i] = to_cdd(make_double2(c, s));
    t32[i] = make_float2((float)c, (float)s);
}

// the tuner's accuracy check: copy every instance's output into one buffer
// (ref[off[i] ..]) or compare it with that copy, recording the largest
// per-instance relative L2 difference (a positive float's bits order like it)
__global__ void k_batch_outputs(const Desc* __restrict__ desc, int count, const int64_t* __restrict__ off,
                                float2* __restrict__ ref, int compare, unsigned* __restrict__ worst) {
    __shared__ double s_num[32], s_den[32];
    for (int it = blockIdx.x; it < count; it += gridDim.x) {
        const Desc d = desc[it];
        float2* r = ref + off[it];
        double num = 0.0, den = 0.0;
        for (int64_t i = threadIdx.x; i < d.N; i += blockDim.x) {
            const float2 o = d.out[i];
            if (!compare) {
                r[i] = o;
            } else {
                const double dx = (double)o.x - r[i].x, dy = (double)o.y - r[i].y;
                num += dx * dx + dy * dy;
                den += (double)r[i].x * r[i].x + (double)r[i].y * r[i].y;
            }
        }
        if (!compare) continue;
        for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_down_sync(0xffffffffu, num, o);
            den += __shfl_down_sync(0xffffffffu, den, o);
        }
        if ((threadIdx.x & 31) == 0) { s_num[threadIdx.x >> 5] = num; s_den[threadIdx.x >> 5] = den; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += s_num[w]; b += s_den[w]; }
            const float rel = b > 0.0 ? (float)sqrt(a / b) : (a > 0.0 ? 1e30f : 0.f);
            atomicMax(worst, __float_as_uint(rel));
        }
        __syncthreads();
    }
}

size_t scratch_bytes(int64_t N, int log_ns, int log_m) {
    const size_t ns = (size_t)1 << log_ns, M = (size_t)1 << log_m;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t s = 0;
    s += al(8 * N) + al(4 * N) + al(8 * N) + al(4 * N) + 2 * al(4 * (ns + 1));
    s += 2 * al(16 * N) + al(16 * kMaxEta * N) + al(16 * kMaxEta * ns) + al(16 * ns);
    s += 2 * al(16 * M) + 2 * al(16 * N) + al(16 * N) + 3 * al(16 * M);
    s += al(8 * N) + 3 * al(8 * M) + 2 * al(8 * N) + 2 * al(8 * ns) + 2 * al(8 * M);
    s += al(8 * N) + al(4 * N);   // node fractions in double-float and float32
    return s;
}

int ceil_log2(int64_t v) {
    int l = 0;
    while (((int64_t)1 << l) < v) ++l;
    return l;
}

}  // namespace
}  // namespace nufft45

using namespace nufft45;

struct nufft_batch_s {
    int count = 0;
    Desc* desc = nullptr;            // device
    int* counter = nullptr;
    int* status = nullptr;
    char* scratch = nullptr;
    size_t scratch_per_cta = 0;
    cdd* twdd = nullptr;
    float2* tw32 = nullptr;
    double* dec_plan = nullptr;
    float* dec_solve = nullptr;
    int grid = 0, threads = 0, max_rl = 3;
    int sms = 1;
    size_t scratch_cap = 0;          // CTAs the scratch slab can hold
    double tol = 0;
    int64_t key_total = 0, key_max = 0;
    // the method's parameters (Sec. V) and the deconvolution tables of the widths
    double gamma = 60.0;
    int eta = 4, w_plan = 14, w_solve = 8;
    std::map<int, int64_t> tab_off;  // log2 grid -> offset in the tables
    int64_t tab_total = 0;
    int tab_w_plan = 0, tab_w_solve = 0;
    int64_t* out_off = nullptr;      // device: first output slot of each descriptor in a packed copy
    int64_t total_n = 0;
};

namespace {
// autotuner cache: (count, sum N, max N, tol) -> (CTAs, threads, radix, gamma, eta, w_plan, w_solve)
struct TuneChoice {
    int grid, threads, max_rl;
    double gamma;
    int eta, w_plan, w_solve;
};
std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int64_t, int64_t, double>, TuneChoice> g_tune;

// Sec. V, Eq. 49: the truncation of the log-kernel series leaves about
// 0.4 gamma^-eta (measured law); the float32 transforms' round-off grows with
// gamma (their rho^{+-k} scalings), about 0.5 gamma 2^-24.
double batch_trunc(double gamma, int eta) { return 0.4 * std::pow(gamma, -eta); }
double batch_roundoff(double gamma) { return 0.5 * gamma * 5.96e-8; }

// default parameters for tol: gamma = 60 with the smallest eta that puts the
// truncation below tol/10, plan width 14 below tol 1e-4 (12 above), width 8
// for the transforms below tol 1e-3 (6 above)
void batch_default_params(double tol, nufft_batch_s* b) {
    b->gamma = 60.0;
    int eta = 1;
    while (eta < kMaxEta && batch_trunc(b->gamma, eta) > tol / 10) ++eta;
    b->eta = eta;
    b->w_plan = tol < 1e-4 ? 14 : 12;
    b->w_solve = tol < 1e-3 ? 8 : 6;
}

// deconvolution tables (1/phihat per grid, centred index) for the current widths
nufft_status batch_tables(nufft_batch_s* b, cudaStream_t s) {
    if (b->tab_w_plan == b->w_plan && b->tab_w_solve == b->w_solve) return NUFFT_OK;
    GLRule glp, gls;
    gauss_legendre_half(2 + (3 * b->w_plan) / 2 + 4, glp);
    gauss_legendre_half(2 + (3 * b->w_solve) / 2 + 4, gls);
    for (auto& kv : b->tab_off) {
        const int64_t ns = (int64_t)1 << kv.first;
        launch_table(KernelShape{b->w_plan, 2.30 * b->w_plan}, glp, ns, ns / 2, ns, 0.0, 0, ns,
                     b->dec_plan + kv.second, nullptr, s);
        launch_table(KernelShape{b->w_solve, 2.30 * b->w_solve}, gls, ns, ns / 2, ns, 0.0, 0, ns, nullptr,
                     b->dec_solve + kv.second, s);
    }
    NUFFT_CUDA_TRY(cudaGetLastError());
    b->tab_w_plan = b->w_plan;
    b->tab_w_solve = b->w_solve;
    return NUFFT_OK;
}
}

extern "C" {

nufft_status nufft_batch_create(int64_t count, const nufft_instance_t* inst, double tol, nufft_stream_t stream,
                                nufft_batch_t* out) {
    if (!out) return fail(NUFFT_ERR_ARG, "null batch output pointer");
    *out = nullptr;
    if (count < 1 || count > (1 << 24)) return fail(NUFFT_ERR_ARG, "count %lld out of range", (long long)count);
    if (!inst) return fail(NUFFT_ERR_ARG, "null instance array");
    if (!(tol >= 1e-6) || tol > 0.1) return fail(tol < 1e-6 && tol > 0 ? NUFFT_ERR_ACCURACY : NUFFT_ERR_ARG,
                                                 "batched tol %g outside [1e-6, 0.1]", tol);
    {
        nufft_status e = cis_table_ensure();   // before any graph capture of the batch kernel
        if (e != NUFFT_OK) return e;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Desc> h(count);
    std::vector<int64_t> order(count);
    for (int64_t i = 0; i < count; ++i) {
        const nufft_instance_t& q = inst[i];
        if (q.N < 2 || q.N > 16384) return fail(NUFFT_ERR_ARG, "instance %lld: N = %lld outside [2, 16384]",
                                                (long long)i, (long long)q.N);
        if (!q.x || !q.in || !q.out) return fail(NUFFT_ERR_ARG, "instance %lld: null pointer", (long long)i);
        if (q.kind != 4 && q.kind != 5) return fail(NUFFT_ERR_ARG, "instance %lld: kind must be 4 or 5", (long long)i);
        order[i] = i;
    }
    // largest instances first: the work queue then balances the tail
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return inst[a].N > inst[b].N; });
    std::map<int, int64_t> tab_off;   // log_ns -> table offset
    int64_t tab_total = 0;
    size_t scratch = 0;
    std::vector<int64_t> off(count);   // packed output offsets, descriptor order
    int64_t total_n = 0;
    for (int64_t i = 0; i < count; ++i) {
        const nufft_instance_t& q = inst[order[i]];
        Desc& d = h[i];
        d.N = q.N;
        d.x = q.x;
        d.in = (const float2*)q.in;
        d.out = (float2*)q.out;
        d.kind = q.kind;
        d.log_ns = std::max(ceil_log2(2 * q.N), ceil_log2(2 * kMaxW));
        d.pow2 = (q.N & (q.N - 1)) == 0;
        d.log_m = d.pow2 ? ceil_log2(q.N) : ceil_log2(2 * q.N - 1);
        d.slot = order[i];
        if (!tab_off.count(d.log_ns)) { tab_off[d.log_ns] = tab_total; tab_total += (int64_t)1 << d.log_ns; }
        d.tab = tab_off[d.log_ns];
        scratch = std::max(scratch, scratch_bytes(d.N, d.log_ns, d.log_m));
        off[i] = total_n;
        total_n += q.N;
    }
    nufft_batch_s* b = new nufft_batch_s();
    b->count = (int)count;
    b->tol = tol;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->sms = std::max(1, sms);
    b->grid = b->sms;
    b->threads = 512;
    b->scratch_per_cta = (scratch + 4095) & ~(size_t)4095;
    b->scratch_cap = (size_t)b->sms * 3;   // room for up to three CTAs per SM
    int64_t tot = 0, mx = 0;
    for (int64_t i = 0; i < count; ++i) { tot += inst[i].N; mx = std::max<int64_t>(mx, inst[i].N); }
    b->key_total = tot;
    b->key_max = mx;
    b->total_n = total_n;
    b->tab_off = tab_off;
    b->tab_total = tab_total;
    batch_default_params(tol, b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(std::make_tuple((int64_t)count, tot, mx, tol));
        if (it != g_tune.end()) {
            const TuneChoice& c = it->second;
            b->grid = c.grid; b->threads = c.threads; b->max_rl = c.max_rl;
            b->gamma = c.gamma; b->eta = c.eta; b->w_plan = c.w_plan; b->w_solve = c.w_solve;
        }
    }
    auto cleanup = [&](nufft_status st) { nufft_batch_destroy(b); return st; };
    cudaError_t e;
    if ((e = cudaMalloc(&b->desc, sizeof(Desc) * count)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMalloc(&b->counter, sizeof(int))) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMalloc(&b->status, sizeof(int) * count)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMalloc(&b->scratch, b->scratch_per_cta * b->scratch_cap)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMalloc(&b->twdd, sizeof(cdd) << kMaxLog)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMalloc(&b->tw32, sizeof(float2) << kMaxLog)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMalloc(&b->dec_plan, sizeof(double) * tab_total)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMalloc(&b->dec_solve, sizeof(float) * tab_total)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMalloc(&b->out_off, sizeof(int64_t) * count)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc", __FILE__, __LINE__));
    if ((e = cudaMemcpyAsync(b->desc, h.data(), sizeof(Desc) * count, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__));
    if ((e = cudaMemcpyAsync(b->out_off, off.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__));
    {
        Launch L(s, K_PLAN_TABLE, 24.0 * (1 << kMaxLog));
        k_twiddle_table<<<(1 << kMaxLog) / 256, 256, 0, s>>>(kMaxLog, b->twdd, b->tw32);
    }
    // deconvolution tables per grid, indexed by the centred index k' + ns/2
    {
        nufft_status ts = batch_tables(b, s);
        if (ts != NUFFT_OK) return cleanup(ts);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup(cuda_fail(e, "table launch", __FILE__, __LINE__));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cleanup(cuda_fail(e, "batch set-up", __FILE__, __LINE__));
    *out = b;
    return NUFFT_OK;
}

nufft_status nufft_batch_run(nufft_batch_t b, nufft_stream_t stream) {
    if (!b) return fail(NUFFT_ERR_ARG, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    NUFFT_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int), s));
    NUFFT_CUDA_TRY(cudaMemsetAsync(b->status, 0, sizeof(int) * b->count, s));
    Args a;
    a.desc = b->desc;
    a.count = b->count;
    a.counter = b->counter;
    a.status = b->status;
    a.scratch = b->scratch;
    a.scratch_per_cta = b->scratch_per_cta;
    a.twdd = b->twdd;
    a.tw32 = b->tw32;
    a.dec_plan = b->dec_plan;
    a.dec_solve = b->dec_solve;
    a.beta_plan = 2.30 * b->w_plan;
    a.beta_solve = 2.30 * b->w_solve;
    a.max_rl = b->max_rl;
    a.gamma = b->gamma;
    a.eta = b->eta;
    a.w_plan = b->w_plan;
    a.w_solve = b->w_solve;
    if (b->tab_w_plan != b->w_plan || b->tab_w_solve != b->w_solve)
        return fail(NUFFT_ERR_ARG, "batch tables do not match its widths");
    {
        Launch L(s, K_PLAN_STAGE, 0.0);
        k_batch<<<b->grid, b->threads, 0, s>>>(a);
    }
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

// Autotuner.  First the launch shape: every (CTAs per SM, threads per CTA,
// largest FFT radix) candidate is timed with CUDA events at the current
// parameters.  Then the method's parameters (Sec. V): candidate sets
// (gamma, eta, plan width, transforms' width) whose a-priori error --
// truncation 0.4 gamma^-eta (Eq. 49's law) within tol/10 and round-off
// 0.5 gamma 2^-24 within tol/2 -- qualifies are run on this batch; a set is
// accepted when every instance's output stays within tol/2 (relative L2) of
// the output of the tightest set (gamma 60, eta 4, widths 14 and 8), and the
// fastest accepted set is kept.  Choices are cached per (count, sum N,
// max N, tol).  The batch's outputs are overwritten.
nufft_status nufft_batch_tune(nufft_batch_t b, nufft_stream_t stream, double* best_ms) {
    if (!b) return fail(NUFFT_ERR_ARG, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    NUFFT_CUDA_TRY(cudaEventCreate(&e0));
    NUFFT_CUDA_TRY(cudaEventCreate(&e1));
    auto time_run = [&](float* ms) -> nufft_status {
        nufft_status st = nufft_batch_run(b, stream);   // warm
        if (st != NUFFT_OK) return st;
        cudaEventRecord(e0, s);
        if ((st = nufft_batch_run(b, stream)) != NUFFT_OK) return st;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return cuda_fail(cudaGetLastError(), "tuner", __FILE__, __LINE__);
        cudaEventElapsedTime(ms, e0, e1);
        return NUFFT_OK;
    };
    float best = 1e30f;
    int bg = b->grid, bt = b->threads, br = b->max_rl;
    nufft_status st = NUFFT_OK;
    for (int per_sm = 1; per_sm <= 3 && st == NUFFT_OK; ++per_sm)
        for (int th : {256, 512})
            for (int rl : {2, 3}) {
                b->grid = b->sms * per_sm;
                b->threads = th;
                b->max_rl = rl;
                float ms = 0.f;
                if ((st = time_run(&ms)) != NUFFT_OK) break;
                if (ms < best) { best = ms; bg = b->grid; bt = th; br = rl; }
            }
    b->grid = bg;
    b->threads = bt;
    b->max_rl = br;
    // the method's parameters, validated on this batch against the tightest set
    struct Cand { double gamma; int eta, w_plan, w_solve; };
    const Cand ref{60.0, 4, 14, 8};
    const Cand cands[] = {{100.0, 3, 12, 8}, {100.0, 3, 10, 8}, {60.0, 4, 12, 8}, {30.0, 4, 12, 8},
                          {60.0, 3, 12, 8}, {300.0, 2, 12, 8}, {100.0, 2, 12, 8}, {100.0, 3, 12, 6}};
    const Cand keep{b->gamma, b->eta, b->w_plan, b->w_solve};
    float2* refout = nullptr;
    unsigned* worst = nullptr;
    Cand bestc = keep;
    if (st == NUFFT_OK) {
        cudaError_t ce = cudaMalloc(&refout, sizeof(float2) * (size_t)b->total_n);
        if (ce == cudaSuccess) ce = cudaMalloc(&worst, sizeof(unsigned));
        if (ce != cudaSuccess) st = cuda_fail(ce, "cudaMalloc", __FILE__, __LINE__);
    }
    auto set = [&](const Cand& c) -> nufft_status {
        b->gamma = c.gamma; b->eta = c.eta; b->w_plan = c.w_plan; b->w_solve = c.w_solve;
        return batch_tables(b, s);
    };
    if (st == NUFFT_OK && (st = set(ref)) == NUFFT_OK) {
        float ms = 0.f;
        if ((st = time_run(&ms)) == NUFFT_OK) {
            k_batch_outputs<<<std::min(b->count, 4 * b->sms), 256, 0, s>>>(b->desc, b->count, b->out_off, refout, 0,
                                                                           worst);
            best = ms;
            bestc = ref;
        }
    }
    for (const Cand& c : cands) {
        if (st != NUFFT_OK) break;
        if (batch_trunc(c.gamma, c.eta) > b->tol / 10 || batch_roundoff(c.gamma) > b->tol / 2) continue;
        if (c.w_solve < 8 && b->tol < 1e-3) continue;
        if ((st = set(c)) != NUFFT_OK) break;
        float ms = 0.f;
        if ((st = time_run(&ms)) != NUFFT_OK) break;
        unsigned w = 0;
        cudaMemsetAsync(worst, 0, sizeof(unsigned), s);
        k_batch_outputs<<<std::min(b->count, 4 * b->sms), 256, 0, s>>>(b->desc, b->count, b->out_off, refout, 1, worst);
        cudaMemcpyAsync(&w, worst, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) { st = cuda_fail(cudaGetLastError(), "tuner", __FILE__, __LINE__); break; }
        float rel = 0.f;
        std::memcpy(&rel, &w, sizeof(rel));
        if (rel <= b->tol / 2 && ms < best) { best = ms; bestc = c; }
    }
    cudaFree(refout);
    cudaFree(worst);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    nufft_status st2 = set(st == NUFFT_OK ? bestc : keep);
    if (st != NUFFT_OK) return st;
    if (st2 != NUFFT_OK) return st2;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[std::make_tuple((int64_t)b->count, b->key_total, b->key_max, b->tol)] =
            TuneChoice{b->grid, b->threads, b->max_rl, b->gamma, b->eta, b->w_plan, b->w_solve};
    }
    if (best_ms) *best_ms = best;
    return NUFFT_OK;
}

nufft_status nufft_batch_params(nufft_batch_t b, nufft_params_t* params) {
    if (!b || !params) return fail(NUFFT_ERR_ARG, "null argument");
    params->gamma = b->gamma;
    params->eta = b->eta;
    params->w_plan = b->w_plan;
    params->w_solve = b->w_solve;
    return NUFFT_OK;
}

nufft_status nufft_batch_config(nufft_batch_t b, int* ctas, int* threads, int* max_radix) {
    if (!b) return fail(NUFFT_ERR_ARG, "null batch");
    if (ctas) *ctas = b->grid;
    if (threads) *threads = b->threads;
    if (max_radix) *max_radix = 1 << b->max_rl;
    return NUFFT_OK;
}

nufft_status nufft_batch_status(nufft_batch_t b, int* status, nufft_stream_t stream) {
    if (!b || !status) return fail(NUFFT_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    NUFFT_CUDA_TRY(cudaMemcpyAsync(status, b->status, sizeof(int) * b->count, cudaMemcpyDefault, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}

nufft_status nufft_batch_destroy(nufft_batch_t b) {
    if (!b) return NUFFT_OK;
    cudaFree(b->desc);
    cudaFree(b->counter);
    cudaFree(b->status);
    cudaFree(b->scratch);
    cudaFree(b->twdd);
    cudaFree(b->tw32);
    cudaFree(b->dec_plan);
    cudaFree(b->dec_solve);
    cudaFree(b->out_off);
    delete b;
    return NUFFT_OK;
}

}  // extern "C"

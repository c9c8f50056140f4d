// Plan-stage kernels (float64): deconvolution and scaling tables, the fold of
// the log-kernel spectrum, kernel samples, Lagrange-kernel coefficients and
// node weights (Secs. III-C to III-E).
#include "internal.h"
#include "cis64.cuh"
#include "df.cuh"

#include <cmath>

namespace nufft45 {

namespace {

constexpr int kTB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)((n + kTB - 1) / kTB); }

// Fourier transform of the spreading kernel at xi cycles per grid step:
//   phihat(xi) = int phi(2x/w) e^{-j 2 pi xi x} dx = w int_0^1 phi(z) cos(pi w xi z) dz,
// by Gauss-Legendre quadrature (the integrand is even in z).
__device__ double phihat(double xi, int w, double beta, const GLRule& gl) {
    double acc = 0.0;
    for (int i = 0; i < gl.nq; ++i) {
        const double z = gl.z[i];
        const double ph = exp(beta * (sqrt(1.0 - z * z) - 1.0));
        acc += gl.wq[i] * ph * cospi(w * xi * z);
    }
    return w * acc;
}

// mode 0: 1/phihat; 1: rho^k/phihat; 2: rho^-k/(P phihat); 3: Lambda_k/phihat with
// Lambda_k = -rho^k/k (Lambda_0 = 0, Eq. 41); 4: rho^k; 5: rho^-k/P;
// 6: Lambda_k / phihat((k mod P) - K0), the fold of Eq. 7 over k = P r + m
__global__ void k_table(int w, double beta, GLRule gl, int64_t n, int64_t K0, int64_t M, double log_rho, int mode,
                        int64_t P, double* out_d, float* out_f) {
    pdl_wait();
    pdl_trigger();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    double v;
    if (mode == 4) v = exp((double)k * log_rho);
    else if (mode == 5) v = exp(-(double)k * log_rho) / (double)P;
    else if (mode == 6) {
        const double ph = phihat((double)(k % P - K0) / (double)n, w, beta, gl);
        v = k == 0 ? 0.0 : -exp((double)k * log_rho) / ((double)k * ph);
    } else {
        const double ph = phihat((double)(k - K0) / (double)n, w, beta, gl);
        if (mode == 0) v = 1.0 / ph;
        else if (mode == 1) v = exp((double)k * log_rho) / ph;
        else if (mode == 2) v = exp(-(double)k * log_rho) / ((double)P * ph);
        else v = k == 0 ? 0.0 : -exp((double)k * log_rho) / ((double)k * ph);
    }
    if (out_d) out_d[k] = v;
    if (out_f) out_f[k] = (float)v;
}

// The node-dependent phases of the plan, one thread per sorted slot i, node
// p = sperm[i]: modp_srt[i] = m = e^{+j 2 pi K0 t_p}; beta[p] =
// e^{-j 2 pi P t_p}; and on each extended slot e that holds p (the middle copy
// at pre + i, the copy shifted by -n if p lies in the last h cells, the copy
// shifted by +n if it lies in the first h cells) conj(m) and the strengths of
// the log-kernel type-1 weighted by it, sx[r][e] = beta^r conj(m), r < eta
// (Eqs. 13, 19, 28), formed in double-float from the two exact-turn phases
__global__ void k_node_phases(const uint64_t* __restrict__ T, const int* __restrict__ sperm,
                              const int* __restrict__ start, int64_t n, int h, int64_t N, uint64_t K0, uint64_t P,
                              int eta, double2* __restrict__ modm_ext, double2* __restrict__ modp_srt,
                              double2* __restrict__ beta, cdd* __restrict__ sx) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int p = sperm[i];
    const uint64_t t = T[p];
    const double2 m = cis_turns_t(K0 * t, +1);
    const double2 b = cis_turns_t(P * t, -1);
    modp_srt[i] = m;
    beta[p] = b;
    const double2 mc = make_double2(m.x, -m.y);
    const int last = start[n - h], pre = start[n] - last, post = start[h];
    int64_t e[3];
    int ne = 0;
    e[ne++] = pre + i;
    if (i >= last) e[ne++] = i - last;
    if (i < post) e[ne++] = pre + N + i;
    cdd v, bd;
    v.x = dd_from_double(mc.x);
    v.y = dd_from_double(mc.y);
    bd.x = dd_from_double(b.x);
    bd.y = dd_from_double(b.y);
    for (int k = 0; k < ne; ++k) modm_ext[e[k]] = mc;
    for (int r = 0; r < eta; ++r) {
        for (int k = 0; k < ne; ++k) sx[(int64_t)r * 2 * N + e[k]] = v;
        v = cmul(v, bd);
    }
}

// Eq. 7 with Lambda = g's coefficients (Eq. 41), the deconvolution folded in:
//   Y_m = sum_{r < eta} fac[P r + m] B_r[(m - K0) mod n],
// B_r the spectrum of the strengths e^{-j 2 pi P r t_p} (grid n)
__global__ void k_fold(const double2* __restrict__ B, int64_t n, int64_t K0, const double* __restrict__ fac,
                       int64_t P, int eta, double2* __restrict__ Y) {
    pdl_wait();
    pdl_trigger();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= P) return;
    double2 acc = make_double2(0.0, 0.0);
    const int64_t src = imod(m - K0, n);
    for (int r = 0; r < eta; ++r) {
        const int64_t k = P * r + m;
        const double2 b = B[r * n + src];
        const double f = fac[k];
        acc.x = fma(f, b.x, acc.x);
        acc.y = fma(f, b.y, acc.y);
    }
    Y[m] = acc;
}

// Eq. 29: K_q = exp(j P pi + j 2 pi sum_p t_p + v_q).  The constant phase is the
// exact turn count P 2^63 + sum T_p mod 2^64.
// K is written in float64 and copied where given: Kf (float32 solves), Kd and
// Kv (the solve's float64 copy, the input of the DFT of Eq. 43)
__global__ void k_kernel_samples(const double2* __restrict__ v, int64_t P, const unsigned long long* __restrict__ sumT,
                                 double2* __restrict__ K, float2* __restrict__ Kf, double2* __restrict__ Kd,
                                 double2* __restrict__ Kv) {
    pdl_wait();
    pdl_trigger();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    const uint64_t C = (uint64_t)*sumT + (uint64_t)P * 0x8000000000000000ull;
    const double2 vq = v[q];
    // the phase in exact 64-bit turns: v's argument taken mod 1 turn, plus C
    double tv = vq.y * 0.15915494309189535;   // 1 / (2 pi)
    tv -= floor(tv);
    const uint64_t Tv = tv < 1.0 ? __double2ull_rz(tv * 18446744073709551616.0) : 0ull;
    const double2 e = cis_turns_t(Tv + C, +1);
    const double mag = exp_t(vq.x);
    const double2 k = make_double2(mag * e.x, mag * e.y);
    K[q] = k;
    if (Kf) Kf[q] = make_float2((float)k.x, (float)k.y);
    if (Kd) Kd[q] = k;
    if (Kv) Kv[q] = k;
}

// Eq. 43 and Eq. 16: L_m = (F_m - P rho^P delta_m) rho^{-m} / P, L_P = 1, and
// the coefficients d_m = (m + 1) L_{m+1} of L', placed on the grid of size n
// for the type-2 that evaluates L'(z_p): grid slot g holds the centred index
// k' = g (g < n - K0) or g - n, m = k' + K0, d_m fac[m] for 0 <= m < P and 0
// elsewhere; rho_neg[m] = rho^{-m}/P (k = m + 1 >= 1: no delta term)
__global__ void k_lcoef_place(const double2* __restrict__ F, int64_t P, const double* __restrict__ rho_neg,
                              int64_t K0, const double* __restrict__ fac, int64_t n, double2* __restrict__ grid) {
    pdl_wait();
    pdl_trigger();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int64_t kc = g < n - K0 ? g : g - n;
    const int64_t m = kc + K0;
    double2 v = make_double2(0.0, 0.0);
    if (m >= 0 && m < P) {
        const int64_t k = m + 1;
        double2 L = make_double2(1.0, 0.0);
        if (k < P) {
            const double2 f = F[k];
            L = make_double2(f.x * rho_neg[k], f.y * rho_neg[k]);
        }
        const double sc = (double)k * fac[m];
        v = make_double2(sc * L.x, sc * L.y);
    }
    grid[g] = v;
}

// The coefficients L_0 .. L_P of Eq. 43 (L_P = 1) zero-padded to n >= 2P, for
// the linear-convolution form of the middle stage
__global__ void k_lagrange_pad(const double2* __restrict__ F, int64_t P, double rhoP, const double* __restrict__ rho_neg,
                               int64_t n, double2* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double2 L = make_double2(0.0, 0.0);
    if (m == P) {
        L.x = 1.0;
    } else if (m < P) {
        double2 f = F[m];
        if (m == 0) f.x -= (double)P * rhoP;   // the delta term of Eq. 43
        L = make_double2(f.x * rho_neg[m], f.y * rho_neg[m]);
    }
    out[m] = L;
}

template <typename TS>
__global__ void k_to_solve(const double2* __restrict__ in, int64_t n, double scale, c2<TS>* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = mk<TS>((TS)(in[i].x * scale), (TS)(in[i].y * scale));
}

// Eqs. 27 / 40: w_p = h(-P t_p + j P a) / (L'(z_p) z_p) with
// h(-P t + j P a) = 1/(rho^P e^{-j 2 pi P t} - 1), one thread per sorted slot
// i (p = sperm[i] visits every node once): w64[p]; the solve-precision slot
// arrays of the sorted list, srt_mod[i] = m = e^{+j 2 pi K0 t_p} (modp_srt) and
// srt_wmod[i] = w_p m; and those of each extended slot e holding p (the middle
// copy at pre + i, the copy of the last h cells, the copy of the first h cells),
// ext_mod[e] = conj(m) and ext_wmod[e] = w_p conj(m).
// (beta, when given, holds e^{-j 2 pi N t_p} by node: the plan's strengths for r = 1)
template <typename TS>
__global__ void k_weights(const uint64_t* __restrict__ T, const int* __restrict__ sperm,
                          const int* __restrict__ start, int64_t n, int h, const double2* __restrict__ D,
                          const double2* __restrict__ modp_srt, const double2* __restrict__ beta, int64_t N,
                          double rhoP, double2* __restrict__ w64, c2<TS>* __restrict__ srt_mod,
                          c2<TS>* __restrict__ srt_wmod, c2<TS>* __restrict__ ext_mod, c2<TS>* __restrict__ ext_wmod) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int p = sperm[i];
    const uint64_t t = T[p];
    const double2 e = beta ? beta[p] : cis_turns_t((uint64_t)N * t, -1);
    const double2 z = cis_turns_t(t, +1);
    const double2 hh = make_double2(rhoP * e.x - 1.0, rhoP * e.y);
    const double2 den = cmul(hh, cmul(D[p], z));
    const double inv = 1.0 / (den.x * den.x + den.y * den.y);
    const double2 w = make_double2(den.x * inv, -den.y * inv);
    w64[p] = w;
    const double2 m = modp_srt[i];
    const double2 wm = cmul(w, m);
    srt_mod[i] = mk<TS>((TS)m.x, (TS)m.y);
    srt_wmod[i] = mk<TS>((TS)wm.x, (TS)wm.y);
    // conj(m) and w conj(m) = conj(conj(w) m) on the extended copies
    const double2 wcm = cmul(w, make_double2(m.x, -m.y));
    const c2<TS> em = mk<TS>((TS)m.x, (TS)-m.y), ewm = mk<TS>((TS)wcm.x, (TS)wcm.y);
    const int last = start[n - h], pre = start[n] - last, post = start[h];
    ext_mod[pre + i] = em;
    ext_wmod[pre + i] = ewm;
    if (i >= last) {
        ext_mod[i - last] = em;
        ext_wmod[i - last] = ewm;
    }
    if (i < post) {
        ext_mod[pre + N + i] = em;
        ext_wmod[pre + N + i] = ewm;
    }
}

}  // namespace

void gauss_legendre_half(int nq, GLRule& r) {
    // nodes/weights of the 2nq-point Gauss-Legendre rule on [-1,1], keeping the
    // nq positive nodes: int_0^1 f = sum w_i f(z_i) for even f.  Newton's
    // method on P_{2nq} from the Chebyshev-like initial guesses.
    const int n2 = 2 * nq;
    r.nq = nq;
    for (int i = 0; i < nq; ++i) {
        double x = std::cos(M_PI * (i + 0.75) / (n2 + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n2; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n2 * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        // recompute derivative at the converged node
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n2; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n2 * (x * p1 - p0) / (x * x - 1.0);
        r.z[i] = x;
        r.wq[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

void launch_table(KernelShape ks, const GLRule& gl, int64_t n, int64_t K0, int64_t M, double log_rho, int mode,
                  int64_t P, double* out_d, float* out_f, cudaStream_t s) {
    Launch L(s, K_PLAN_TABLE, M * (out_d ? 8.0 : 4.0));
    launch_k(k_table, nblk(M), kTB, 0, s, ks.w, ks.beta, gl, n, K0, M, log_rho, mode, P, out_d, out_f);
}

void launch_node_phases(const uint64_t* T, const Geometry& g, uint64_t K0, uint64_t P, int eta, double2* modm_ext,
                        double2* modp_srt, double2* beta, void* sx, cudaStream_t s) {
    const int64_t N = g.N;
    Launch L(s, K_PLAN_STAGE, N * (4.0 + 8.0 + 16.0 + 16.0) + 2.0 * N * (16.0 + 16.0 * eta));
    launch_k(k_node_phases, nblk(N), kTB, 0, s, T, g.srt_perm, g.cell_start, g.n, g.w / 2, N, K0, P, eta, modm_ext,
             modp_srt, beta, static_cast<cdd*>(sx));
}

void launch_fold(const double2* B, int64_t n, int64_t K0, const double* fac, int64_t P, int eta, double2* Y,
                 cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, (double)eta * P * 24.0 + P * 16.0);
    launch_k(k_fold, nblk(P), kTB, 0, s, B, n, K0, fac, P, eta, Y);
}

void launch_kernel_samples(const double2* v, int64_t P, const unsigned long long* sumT, double2* K, float2* Kf,
                           double2* Kd, double2* Kv, cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, P * (32.0 + (Kf ? 8.0 : 0.0) + (Kd ? 16.0 : 0.0) + (Kv ? 16.0 : 0.0)));
    launch_k(k_kernel_samples, nblk(P), kTB, 0, s, v, P, sumT, K, Kf, Kd, Kv);
}

void launch_lcoef_place(const double2* F, int64_t P, const double* rho_neg, int64_t K0, const double* fac, int64_t n,
                        double2* grid, cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, P * 32.0 + n * 16.0);
    launch_k(k_lcoef_place, nblk(n), kTB, 0, s, F, P, rho_neg, K0, fac, n, grid);
}

void launch_lagrange_pad(const double2* F, int64_t P, double rhoP, const double* rho_neg, int64_t n, double2* out,
                         cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, P * 24.0 + n * 16.0);
    launch_k(k_lagrange_pad, nblk(n), kTB, 0, s, F, P, rhoP, rho_neg, n, out);
}

template <typename TS>
void launch_to_solve(const double2* in, int64_t n, double scale, c2<TS>* out, cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, n * (16.0 + sizeof(c2<TS>)));
    launch_k(k_to_solve<TS>, nblk(n), kTB, 0, s, in, n, scale, out);
}
template void launch_to_solve<float>(const double2*, int64_t, double, float2*, cudaStream_t);
template void launch_to_solve<double>(const double2*, int64_t, double, double2*, cudaStream_t);

template <typename TS>
void launch_weights(const uint64_t* T, const Geometry& g, const double2* D, const double2* modp_srt,
                    const double2* beta, double rhoP, double2* w64, c2<TS>* wt2_srt, c2<TS>* wt4_srt,
                    c2<TS>* wt1_ext, c2<TS>* wt5_ext, cudaStream_t s) {
    const int64_t N = g.N;
    Launch L(s, K_PLAN_STAGE, N * (4.0 + 8.0 + 16.0 + 16.0 + 16.0 + (beta ? 16.0 : 0.0) + 12.0 * sizeof(TS)));
    launch_k(k_weights<TS>, nblk(N), kTB, 0, s, T, g.srt_perm, g.cell_start, g.n, g.w / 2, D, modp_srt, beta, N,
             rhoP, w64, wt2_srt, wt4_srt, wt1_ext, wt5_ext);
}
template void launch_weights<float>(const uint64_t*, const Geometry&, const double2*, const double2*,
                                    const double2*, double, double2*, float2*, float2*, float2*, float2*,
                                    cudaStream_t);
template void launch_weights<double>(const uint64_t*, const Geometry&, const double2*, const double2*,
                                     const double2*, double, double2*, double2*, double2*, double2*, double2*,
                                     cudaStream_t);

nufft_status plan_kernels_init() { return cis_table_ensure(); }

namespace {
__global__ void k_debug_cis(const uint64_t* __restrict__ T, int64_t n, double2* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = cis_turns_t(T[i], +1);
}
__global__ void k_debug_exp_t(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = exp_t(x[i]);
}
}  // namespace

}  // namespace nufft45

// Test hook (not part of the public header): out[i] = e^{j 2 pi T[i] / 2^64}
// by the plan kernels' table-driven evaluation; device arrays of n entries.
extern "C" nufft_status nufft_debug_cis(int64_t n, const uint64_t* T, void* out, nufft_stream_t stream) {
    using namespace nufft45;
    if (n < 0 || (n > 0 && (!T || !out))) return fail(NUFFT_ERR_ARG, "bad cis test arguments");
    nufft_status st = plan_kernels_init();
    if (st != NUFFT_OK || n == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    launch_k(k_debug_cis, nblk(n), kTB, 0, s, T, n, static_cast<double2*>(out));
    NUFFT_CUDA_TRY(cudaGetLastError());
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}


// Test hook (not part of the public header): out[i] = e^{x[i]} by the plan
// kernels' table-driven float64 exponential (|x| < 700); device arrays of n.
extern "C" nufft_status nufft_debug_exp64(int64_t n, const double* x, double* out, nufft_stream_t stream) {
    using namespace nufft45;
    if (n < 0 || (n > 0 && (!x || !out))) return fail(NUFFT_ERR_ARG, "bad exp test arguments");
    nufft_status st = plan_kernels_init();
    if (st != NUFFT_OK || n == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    launch_k(k_debug_exp_t, nblk(n), kTB, 0, s, x, n, out);
    NUFFT_CUDA_TRY(cudaGetLastError());
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}

// Plan-stage kernels (float64): deconvolution and scaling tables, the fold of
// the log-kernel spectrum, kernel samples, Lagrange-kernel coefficients and
// node weights (Secs. III-C to III-E).
#include "internal.h"
#include "cis64.cuh"

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

// e^{sign j 2 pi K0 t_p} for p = perm[i], i < count (count read from device when given)
__global__ void k_mod(const uint64_t* __restrict__ T, const int* __restrict__ perm, int64_t cap,
                      const int* __restrict__ count_dev, uint64_t K0, int sign, double2* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cnt = count_dev ? (int64_t)*count_dev : cap;
    if (i >= cnt) return;
    out[i] = cis_turns_t(K0 * T[perm[i]], sign);
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

// strengths of the log-kernel type-1: out[r][p] = e^{-j 2 pi P r t_p}, r < eta
__global__ void k_plan_strengths(const uint64_t* __restrict__ T, int64_t N, uint64_t P, int eta,
                                 double2* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const uint64_t t = T[p];
    for (int r = 0; r < eta; ++r) out[(int64_t)r * N + p] = cis_turns_t(P * (uint64_t)r * t, -1);
}

// Eq. 29: K_q = exp(j P pi + j 2 pi sum_p t_p + v_q).  The constant phase is the
// exact turn count P 2^63 + sum T_p mod 2^64.
__global__ void k_kernel_samples(const double2* __restrict__ v, int64_t P, const unsigned long long* __restrict__ sumT,
                                 double2* __restrict__ K, float2* __restrict__ Kf) {
    pdl_wait();
    pdl_trigger();
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P) return;
    const uint64_t C = (uint64_t)*sumT + (uint64_t)P * 0x8000000000000000ull;
    const double2 vq = v[q];
    double s, c;
    sincospi(vq.y / 3.141592653589793238462643383279502884 + 2.0 * turns_of(C), &s, &c);
    const double mag = exp(vq.x);
    const double2 k = make_double2(mag * c, mag * s);
    K[q] = k;
    if (Kf) Kf[q] = make_float2((float)k.x, (float)k.y);
}

// Eq. 43 and Eq. 16: L_m = (F_m - P rho^P delta_m) rho^{-m} / P, L_P = 1,
// d_m = (m + 1) L_{m+1}; rho_neg[m] = rho^{-m}/P.
__global__ void k_lcoef(const double2* __restrict__ F, int64_t P, double rhoP, const double* __restrict__ rho_neg,
                        double2* __restrict__ d) {
    pdl_wait();
    pdl_trigger();
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= P) return;
    double2 L;
    const int64_t k = m + 1;
    if (k == P) L = make_double2(1.0, 0.0);
    else {
        const double2 f = F[k];
        L = make_double2(f.x * rho_neg[k], f.y * rho_neg[k]);   // k >= 1: no delta term
    }
    d[m] = make_double2((double)k * L.x, (double)k * L.y);
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
// h(-P t + j P a) = 1/(rho^P e^{-j 2 pi P t} - 1).
__global__ void k_weights(const uint64_t* __restrict__ T, const double2* __restrict__ D, int64_t N, double rhoP,
                          double2* __restrict__ w) {
    pdl_wait();
    pdl_trigger();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const uint64_t t = T[p];
    const double2 e = cis_turns_t((uint64_t)N * t, -1);
    const double2 z = cis_turns_t(t, +1);
    const double2 h = make_double2(rhoP * e.x - 1.0, rhoP * e.y);
    const double2 den = cmul(h, cmul(D[p], z));
    const double nn = den.x * den.x + den.y * den.y;
    w[p] = make_double2(den.x / nn, -den.y / nn);
}

// per-slot solve weights: plain modulation e^{sign j 2 pi K0 t} and the node
// weight times it, in the solve precision
template <typename TS>
__global__ void k_slot_weights(const uint64_t* __restrict__ T, const int* __restrict__ perm, int64_t cap,
                               const int* __restrict__ count_dev, uint64_t K0, int sign,
                               const double2* __restrict__ w_user, c2<TS>* __restrict__ mod_out,
                               c2<TS>* __restrict__ wmod_out) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cnt = count_dev ? (int64_t)*count_dev : cap;
    if (i >= cnt) return;
    const int p = perm[i];
    const double2 m = cis_turns_t(K0 * T[p], sign);
    mod_out[i] = mk<TS>((TS)m.x, (TS)m.y);
    const double2 wm = cmul(w_user[p], m);
    wmod_out[i] = mk<TS>((TS)wm.x, (TS)wm.y);
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

void launch_mod(const uint64_t* T, const int* perm, int64_t cap, const int* count_dev, uint64_t K0, int sign,
                double2* out, cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, cap * 28.0);
    launch_k(k_mod, nblk(cap), kTB, 0, s, T, perm, cap, count_dev, K0, sign, out);
}

void launch_fold(const double2* B, int64_t n, int64_t K0, const double* fac, int64_t P, int eta, double2* Y,
                 cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, (double)eta * P * 24.0 + P * 16.0);
    launch_k(k_fold, nblk(P), kTB, 0, s, B, n, K0, fac, P, eta, Y);
}

void launch_plan_strengths(const uint64_t* T, int64_t N, uint64_t P, int eta, double2* out, cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, N * (8.0 + 16.0 * eta));
    launch_k(k_plan_strengths, nblk(N), kTB, 0, s, T, N, P, eta, out);
}

void launch_kernel_samples(const double2* v, int64_t P, const unsigned long long* sumT, double2* K, float2* Kf,
                           cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, P * (Kf ? 40.0 : 32.0));
    launch_k(k_kernel_samples, nblk(P), kTB, 0, s, v, P, sumT, K, Kf);
}

void launch_lcoef(const double2* F, int64_t P, double rhoP, const double* rho_neg, double2* d, cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, P * 40.0);
    launch_k(k_lcoef, nblk(P), kTB, 0, s, F, P, rhoP, rho_neg, d);
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

void launch_weights(const uint64_t* T, const double2* D, int64_t N, double rhoP, double2* w, cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, N * 40.0);
    launch_k(k_weights, nblk(N), kTB, 0, s, T, D, N, rhoP, w);
}

template <typename TS>
void launch_slot_weights(const uint64_t* T, const int* perm, int64_t cap, const int* count_dev, uint64_t K0, int sign,
                         const double2* w_user, c2<TS>* mod_out, c2<TS>* wmod_out, cudaStream_t s) {
    Launch L(s, K_PLAN_STAGE, cap * (28.0 + 4.0 * sizeof(TS)));
    launch_k(k_slot_weights<TS>, nblk(cap), kTB, 0, s, T, perm, cap, count_dev, K0, sign, w_user, mod_out, wmod_out);
}
template void launch_slot_weights<float>(const uint64_t*, const int*, int64_t, const int*, uint64_t, int,
                                         const double2*, float2*, float2*, cudaStream_t);
template void launch_slot_weights<double>(const uint64_t*, const int*, int64_t, const int*, uint64_t, int,
                                          const double2*, double2*, double2*, cudaStream_t);

nufft_status plan_kernels_init() { return cis_table_ensure(); }

namespace {
__global__ void k_debug_cis(const uint64_t* __restrict__ T, int64_t n, double2* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = cis_turns_t(T[i], +1);
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


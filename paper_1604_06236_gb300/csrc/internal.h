// Internal interfaces of the nufft45 library (host side, C++).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "nufft45.h"
#include "common.cuh"

namespace nufft45 {

nufft_status cuda_fail(cudaError_t e, const char* expr, const char* file, int line);
nufft_status fail(nufft_status st, const char* fmt, ...);

// Launch `kern` on stream s as a programmatic dependent of the previous kernel
// in s (see pdl_wait in common.cuh: every kernel of the library waits for its
// predecessor before touching memory).  Errors surface through
// cudaGetLastError like a <<<>>> launch.
template <typename... KArgs, typename... Args>
void launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ------------------------------------------------------------- tracing ----
// Construct around every kernel launch: counts launches and, when tracing is
// on, records events on the launch stream before and after the launch and
// attributes them (and `bytes`, the algorithmic traffic) to a kernel class
// (float64 launches get the class's "_f64" twin).
enum KernelKind { K_FFT = 0, K_SPREAD, K_INTERP, K_SELECT, K_PLACE, K_POINTWISE, K_GEOMETRY, K_PLAN_TABLE,
                  K_PLAN_STAGE, K_BLUESTEIN, K_COUNT };
const char* kind_name(int k);
class Launch {
  public:
    Launch(cudaStream_t s, int kind, double bytes, bool f64 = false);
    ~Launch();
  private:
    cudaStream_t s_;
    int kind_;
    double bytes_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};
// Traces the launches of one unit (the passes of one FFT) that run back to
// back on a stream with one pair of events instead of one pair per launch, so
// that tracing leaves their programmatic overlap intact.  Launches of the
// group's kind on its stream, made on this thread while the group lives, join
// it; a launch of another kind ends the current run of the group (a later
// launch of its kind starts a new one).  Groups nest: an inner group joins the
// outer one.
class LaunchGroup {
  public:
    LaunchGroup(cudaStream_t s, int kind, bool f64 = false);
    ~LaunchGroup();
    bool join(cudaStream_t s, int kind, double bytes);   // called by Launch
    void close();                                        // ends the current run
  private:
    cudaStream_t s_;
    int kind_;
    bool outer_ = false;
    cudaEvent_t a_ = nullptr;
    long long n_ = 0;
    double bytes_ = 0;
};

// ---------------------------------------------------------------- FFT ------
// One Stockham autosort pass of composite radix R: for every j < n/R the R
// inputs x[j + k n/R] are twiddled by W_{Ns R}^{(j mod Ns) k}, transformed by a
// length-R DFT done in shared memory (sub-radices `sub`), and written to
// y[(j/Ns) Ns R + (j mod Ns) + m Ns].  After all passes the output is in
// natural order.
struct FFTPass {
    int R = 1;
    int64_t Ns = 1;
    int nsub = 0;
    int sub[12] = {0};
    int C = 1;          // butterflies (columns) per CTA
};

struct FFTPlan {
    int64_t n = 0;
    int prec = 0;                       // 1 = float, 2 = double, 3 = double-float
    std::vector<FFTPass> passes;
    std::vector<int> p2_rlog;           // power-of-two plan: log2 radix of each pass
    std::vector<int> q_rlog;            // double-float power-of-two plans: passes of the few-vector kernel
    // two-level table of W_n^e = e^{-j 2 pi e / n}: lo[e & (B-1)] * hi[e >> shift]
    int shift = 0;
    void* tw_lo = nullptr;
    void* tw_hi = nullptr;
    void* tw_full = nullptr;            // W_n^e for every e < n (power-of-two plans)
    // Bluestein (n has a prime factor > 7): length-m convolution
    bool bluestein = false;
    int64_t m = 0;
    std::unique_ptr<FFTPlan> sub;
    void* chirp = nullptr;              // e^{+j pi k^2 / n}, k < n
    void* chirp_hat_fwd = nullptr;      // FFT_m of the forward filter, / m
    void* chirp_hat_inv = nullptr;      // FFT_m of the inverse filter, / m
    ~FFTPlan();
};

bool is_smooth(int64_t n);                 // only prime factors 2, 3, 5, 7
int64_t next_smooth(int64_t n);            // smallest smooth m >= n
nufft_status fft_make(FFTPlan& p, int64_t n, int prec, cudaStream_t s);
// scratch elements (complex) fft_exec needs besides its buffer, per batch item
int64_t fft_work_elems(const FFTPlan& p);
// NUFFT_ERR_TIMEOUT if a bounded in-kernel wait of an FFT pass expired since
// the last call (synchronises s, then clears the count), else NUFFT_OK
nufft_status fft_wait_status(cudaStream_t s);
// In-place-by-result: transforms `buf` (batch contiguous items of n) with
// dir = -1 (sum x e^{-j2pi jk/n}) or +1 (sum x e^{+j2pi jk/n}), unnormalised.
// Returns the pointer that holds the result (buf or work).
template <typename T>
nufft_status fft_exec(const FFTPlan& p, c2<T>* buf, c2<T>* work, int64_t batch, int dir,
                      cudaStream_t s, c2<T>** result);
// float64 vectors through a double-float plan (prec 3): ~2^-48 relative
// accuracy with the arithmetic on the float32 pipes.  io bit 1: the input is
// already complex double-float (no conversion); bit 2: leave the result in
// complex double-float.
constexpr int kDdIn = 1, kDdOut = 2;
nufft_status fft_exec_dd(const FFTPlan& p, double2* buf, double2* work, int64_t batch, int dir, cudaStream_t s,
                         double2** result, int io = 0);

// Element-wise work fused into the first pass's loads (lop) and the last
// pass's stores (sop) of a multi-pass power-of-two FFT; idx is the element's
// position in its length-n vector:
//   lop 1: x[idx] = src[b * src_bs + ((idx - K0) mod ns)] * fac_in[idx]
//   lop 2: x[idx] = in[idx] * fac_in[idx]
//   lop 3: the input is known to be zero outside idx < n/4 and idx >= 3n/4
//          (a centred spectrum filling half of the grid): only that half is
//          read, so the rest of `in` need not be cleared
//   sop 1: y[idx] *= mulc[idx];   sop 2: y[idx] *= fac_out[idx]
// and two scattering stores, where `out` has batch stride out_bs:
//   sop 3 (select): k = (idx + K0) mod n; if k < P: out[b out_bs + k] = y[idx] fac_out[k]
//   sop 4 (place):  out[b out_bs + ((idx - K0) mod ns)] = y[idx] fac_out[idx]
struct FFTHooks {
    int lop = 0, sop = 0;
    const void* src = nullptr;
    int64_t src_bs = 0, ns = 0, K0 = 0;
    const void* fac_in = nullptr;
    const void* mulc = nullptr;
    const void* fac_out = nullptr;
    int64_t out_bs = 0, P = 0;
};
template <typename T> bool fft_hooks_supported(const FFTPlan& p);
// the scattering stores (sop 3, 4) run on this plan: float32, two TMA-fed passes
template <typename T> bool fft_scatter_supported(const FFTPlan& p);
// out = FFT_{-dir}( fmul * FFT_{dir}(in) ) for two-pass n = 256 x 256 float32
// plans, in three launches (the middle one runs the first transform's last
// pass, the product and the second transform's first pass); h.lop applies to
// the first loads, h.sop to the last stores; in -> w1 -> w2 -> out
template <typename T> bool fft_conv_supported(const FFTPlan& p);
template <typename T>
nufft_status fft_exec_conv(const FFTPlan& p, const c2<T>* in, c2<T>* w1, c2<T>* w2, c2<T>* out, int64_t batch,
                           int dir, const c2<T>* fmul, const FFTHooks& h, cudaStream_t s);
// in -> out (never writes `in`; `work` and `out` are the ping-pong buffers)
template <typename T>
nufft_status fft_exec_hooked(const FFTPlan& p, const c2<T>* in, c2<T>* work, c2<T>* out, int64_t batch, int dir,
                             const FFTHooks& h, cudaStream_t s);

// ------------------------------------------------------- node geometry ----
// Nodes sorted by cell of a grid of size n (counting sort, ties by index),
// plus the wrapped ("extended") copy used by output-stationary spreading: the
// nodes of the last w/2 cells are prepended with cell - n and those of the
// first w/2 cells appended with cell + n.  Grid point g gathers the extended
// nodes [cstart[g], cstart[g + w]).
struct Geometry {
    int64_t N = 0, n = 0;
    int w = 0;                 // halo width the extended arrays were built for
    int* srt_perm = nullptr;   // sorted slot -> node index                [N]
    int* srt_cell = nullptr;   //                                          [N]
    double* srt_frac = nullptr;  // n t - cell in [0,1)                    [N]
    float* srt_fracf = nullptr;  //                                        [N]
    int* ext_perm = nullptr;   //                                          [2N]
    int* ext_cell = nullptr;   //                                          [2N]
    double* ext_frac = nullptr;  //                                        [2N]
    float* ext_fracf = nullptr;  //                                        [2N]
    int* cstart = nullptr;     // [n + w + 1]
    int* dup_flag = nullptr;   // set when two nodes coincide mod 1
    const int* cell_start = nullptr;   // [n + 1] first sorted slot of each cell (plan scratch: valid while the plan is built)
};

// ------------------------------------------------------------- launchers --
struct KernelShape { int w; double beta; };

// per-device tables the plan kernels read (call before the first plan on a device)
nufft_status plan_kernels_init();

// From the nodes x (radians): the exact turns T, the cell-sorted and extended
// node lists, the duplicate-node flag (cleared, then set when two nodes
// coincide) and sumT = sum of T mod 2^64 (the constant phase of Eq. 29)
nufft_status build_geometry(Geometry& g, const double* x, uint64_t* T, int64_t N, int64_t n, int w,
                            bool want_float, int* scratch_int, unsigned long long* sumT, cudaStream_t s);
int64_t geometry_scratch_ints(int64_t N, int64_t n);

template <typename T>
void launch_spread(const Geometry& g, KernelShape ks, const c2<T>* src, int64_t src_bs,
                   const c2<T>* wt_ext, c2<T>* grid, int64_t batch, cudaStream_t s);
template <typename T>
void launch_interp(const Geometry& g, KernelShape ks, const c2<T>* grid, const c2<T>* wt_srt,
                   c2<T>* dst, int64_t dst_bs, int64_t batch, cudaStream_t s);
// The plan's pair in double-float ("complex double-float": 16 bytes per
// value, real hi, real lo, imaginary hi, imaginary lo): the spread takes
// weighted strengths per extended slot (sx[b sx_bs + slot], batch <= 4 per
// launch row), writes the grid in that format and stores its kernel values as
// double-float pairs in ktab (N * ks.w); the interpolation reads both and
// writes dst[perm[i]] = (sum over taps) * wt[i] in float64.
void launch_spread_plan_dd(const Geometry& g, KernelShape ks, const void* sx, int64_t sx_bs, void* grid,
                           int64_t batch, cudaStream_t s, void* ktab);
void launch_interp_plan_dd(const Geometry& g, KernelShape ks, const void* grid, const void* ktab, const double2* wt,
                           double2* dst, cudaStream_t s);
// float64 type-2 interpolation from a complex double-float grid (batch stride
// n): taps summed in double-float, dst[b dst_bs + perm[i]] = sum * wt_srt[i]
void launch_interp_dd(const Geometry& g, KernelShape ks, const void* grid, const double2* wt_srt, double2* dst,
                      int64_t dst_bs, int64_t batch, cudaStream_t s);

// out[b][k] = in[b][(k - K0) mod n] * fac[k], k < P
template <typename T>
void launch_select(const c2<T>* in, int64_t n, c2<T>* out, int64_t out_bs, int64_t P, int64_t K0,
                   const T* fac, int64_t batch, cudaStream_t s);
// out[b][g] = in[b][k] * fac[k] (* j 2 pi k when deriv) where k = g' + K0 for the
// centred index g' of g, 0 elsewhere
template <typename T>
void launch_place(const c2<T>* in, int64_t in_bs, int64_t P, int64_t K0, const T* fac, c2<T>* out,
                  int64_t n, int64_t batch, cudaStream_t s, bool deriv = false);
// out[b][k] = in[b][k] * (mulc ? mulc[k] : 1) * (fac ? fac[k] : 1)
template <typename T>
void launch_pointwise(const c2<T>* in, int64_t in_bs, c2<T>* out, int64_t out_bs, int64_t P,
                      const c2<T>* mulc, const T* fac, int64_t batch, cudaStream_t s);

// refinement: out = (double) in; r = in - y (float64 difference, stored in T); out += c
template <typename T> void launch_widen(const c2<T>* in, double2* out, int64_t n, cudaStream_t s);
template <typename T> void launch_residual(const c2<T>* in, const double2* y, c2<T>* r, int64_t n, cudaStream_t s);
template <typename T> void launch_accumulate(c2<T>* out, const c2<T>* c, int64_t n, cudaStream_t s);

// out[q] = scale * sum_b Re(conj(X[b][q]) Y[b][q]) (float64 accumulation)
template <typename T>
void launch_grad_nodes(const c2<T>* X, const c2<T>* Y, int64_t N, int64_t batch, double scale, double* out,
                       cudaStream_t s);

// plan-stage kernels (float64)
struct GLRule { int nq; double z[48]; double wq[48]; };
void gauss_legendre_half(int nq, GLRule& r);   // nodes in (0,1), weights for int_0^1 of an even function
// tables over k < M: mode 0: 1/phihat((k-K0)/n); 1: rho^k/phihat; 2: rho^-k/(P phihat);
// 3: Lambda_k/phihat, Lambda_k = -rho^k/k; 4: rho^k; 5: rho^-k/P;
// 6: Lambda_k/phihat((k mod P) - K0)
void launch_table(KernelShape ks, const GLRule& gl, int64_t n, int64_t K0, int64_t M, double log_rho, int mode,
                  int64_t P, double* out_d, float* out_f, cudaStream_t s);
// modp_srt[i] = e^{+j 2 pi K0 t_{sperm[i]}}, i < N, and its conjugate on every
// extended slot of the same node (modm_ext); beta[p] = e^{-j 2 pi P t_p}; the
// plan spread's strengths per extended slot in complex double-float,
// sx[r * 2N + e] = beta^r e^{-j 2 pi K0 t_p}, r < eta
void launch_node_phases(const uint64_t* T, const Geometry& g, uint64_t K0, uint64_t P, int eta, double2* modm_ext,
                        double2* modp_srt, double2* beta, void* sx, cudaStream_t s);
// Y_m = sum_{r<eta} fac[P r + m] B[r n + (m - K0) mod n]
void launch_fold(const double2* B, int64_t n, int64_t K0, const double* fac, int64_t P, int eta, double2* Y,
                 cudaStream_t s);
// K_q (Eq. 29) into K, and copies into Kf (float32), Kd and Kv where not null
void launch_kernel_samples(const double2* v, int64_t P, const unsigned long long* sumT, double2* K, float2* Kf,
                           double2* Kd, double2* Kv, cudaStream_t s);
// d_m = (m + 1) L_{m+1} (Eqs. 43, 16) times fac[m], placed on the grid of size n
// at the centred index m - K0 (0 elsewhere)
void launch_lcoef_place(const double2* F, int64_t P, const double* rho_neg, int64_t K0, const double* fac, int64_t n,
                        double2* grid, cudaStream_t s);
// L_0 .. L_P (Eq. 43) from F = DFT(K), zero-padded to n
void launch_lagrange_pad(const double2* F, int64_t P, double rhoP, const double* rho_neg, int64_t n, double2* out,
                         cudaStream_t s);
template <typename TS>
void launch_to_solve(const double2* in, int64_t n, double scale, c2<TS>* out, cudaStream_t s);
// out[b][m] = c[b][m] + rho^P c[b][m + P], m < P (c of batch stride n)
template <typename T>
void launch_conv_fold(const c2<T>* c, int64_t n, int64_t P, double rhoP, c2<T>* out, int64_t out_bs, int64_t batch,
                      cudaStream_t s);
// w_p (Eqs. 27, 40) into w64 (node order) and the solve-precision slot arrays:
// sorted slots wt2 = e^{+j 2 pi K0 t}, wt4 = w wt2; extended slots
// wt1 = e^{-j 2 pi K0 t}, wt5 = w wt1
// (beta: e^{-j 2 pi N t_p} by node when already at hand, else null; one
// launch: the extended slots are reached from the sorted ones through the
// geometry's cell starts)
template <typename TS>
void launch_weights(const uint64_t* T, const Geometry& g, const double2* D, const double2* modp_srt,
                    const double2* beta, double rhoP, double2* w64, c2<TS>* wt2_srt, c2<TS>* wt4_srt,
                    c2<TS>* wt1_ext, c2<TS>* wt5_ext, cudaStream_t s);

}  // namespace nufft45

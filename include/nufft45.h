/*
 * nufft45.h -- non-iterative inverse nonuniform FFTs of types 4 and 5 in one
 * dimension (J. Selva, "Non-iterative Type 4 and 5 Nonuniform FFT Methods in
 * the One-Dimensional Case"), with the type-1 and type-2 transforms they are
 * built from.  CUDA library for GB300 (sm_103a).
 *
 * Conventions shared by every call
 * ---------------------------------
 * Nodes.  P = N nodes x_p in radians (any real value; wrapped to [0, 2 pi)).
 *   The library uses t_p = x_p / (2 pi) mod 1, carried exactly as the 64-bit
 *   fraction T_p = trunc(t_p 2^64).  Sec. II assumes 0 <= t_p < 1.
 * Frequencies are 0 .. N-1, not centred (Sec. I notation; Eqs. 32, 34).
 * Data.  Interleaved complex: complex64 (float re, im) for NUFFT_FP32 plans,
 *   complex128 (double re, im) for NUFFT_FP64 plans.  `batch` right-hand
 *   sides are contiguous with stride N elements.  Out-of-place only: the
 *   input and output buffers must not overlap.
 * Pointers.  Device pointers, or host pointers (pinned or pageable), staged
 *   through device memory.  Pageable host buffers are copied on `stream` and
 *   the call returns after the result has been copied back.  Pinned host
 *   buffers (page-locked, e.g. cudaHostAlloc) are copied on the library's own
 *   copy streams (one per direction and device), ordered after the work
 *   queued on `stream` by events, so the copies overlap transforms queued
 *   earlier or later: the call returns once the work is queued; the host
 *   input must not change, and the host output is not complete, until
 *   nufft_stream_check(stream) returns or the device is synchronised.  For
 *   device buffers the call is asynchronous on `stream`.  Buffers stay owned
 *   by the caller.
 * Stream.  A cudaStream_t (NULL = legacy default stream).
 * Errors.  Every call returns a status and never aborts or traps; the
 *   message of the last failure on the calling thread is available from
 *   nufft_last_error_message().  Argument errors are reported before any
 *   work is queued.
 */
#ifndef NUFFT45_H
#define NUFFT45_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* nufft_stream_t;   /* the same type as cudaStream_t */
typedef struct nufft_plan_s* nufft_plan_t;    /* opaque */

typedef enum {
    NUFFT_OK = 0,
    NUFFT_ERR_ARG = 1,        /* bad argument (size, pointer, tolerance, precision) */
    NUFFT_ERR_DUP_NODES = 2,  /* two nodes coincide modulo 2 pi: the system of Eq. 47/48 is singular */
    NUFFT_ERR_ALLOC = 3,      /* device memory allocation failed */
    NUFFT_ERR_CUDA = 4,       /* a CUDA runtime call or kernel launch failed */
    NUFFT_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up */
    NUFFT_ERR_ACCURACY = 6    /* the tolerance cannot be met in the requested precision */
} nufft_status;

typedef enum {
    NUFFT_FP32 = 1,   /* node-dependent plan in float64, transforms in float32 (complex64 data) */
    NUFFT_FP64 = 2,   /* everything in float64 (complex128 data) */
    /* OR-ed into the precision: nufft_inv5/nufft_inv4 apply the refined method
     * of Sec. V (R-NFFT): the inverse is applied again to the residual
     * b - F x1, formed by a float64 type-2 (resp. type-1) transform, and the
     * correction is added, taking the relative error from eps to about eps^2
     * (Eqs. 44-46).  For ill-conditioned node sets (near-coincident nodes). */
    NUFFT_REFINE = 0x100,
    /* OR-ed into the precision (no counterpart in the paper): nufft_plan
     * returns as soon as the plan's kernels are enqueued instead of waiting
     * for them to read back the duplicate-node check.  The check still runs
     * on the device; nufft_plan_check reports it.  Device node arrays must
     * then stay valid until the plan's kernels have run (stream order). */
    NUFFT_DEFER_CHECK = 0x200,
    /* OR-ed into the precision: nufft_inv5/nufft_inv4 apply the middle stage
     * (Eqs. 37, 30, 31) in its equivalent linear-convolution form
     * S_m = c_m + rho^P c_{m+P}, c = L * A, with the Lagrange coefficients
     * L_0..L_P of Eq. 43 (no counterpart in the paper's text; it follows from
     * Eqs. 10, 30, 31 by expanding K_q = L(rho e^{j 2 pi q/P})).  The solve then
     * carries no rho^{-m} scaling, whose round-off grows with gamma; it costs
     * two FFTs of the grid size instead of two of size N. */
    NUFFT_TOEPLITZ = 0x400
} nufft_prec;

/*
 * nufft_plan -- precompute everything that depends on the nodes.
 *   Sec. III (Fig. 1, upper half) and Sec. IV: the log-kernel samples v(q/P)
 *   by a type-1 NUFFT of unit strengths of length R = eta P (Eqs. 13, 19, 28,
 *   41, 42, folded by Eq. 7), the kernel samples K_q = L(e^{j 2 pi (q/P + ja)})
 *   (Eq. 29), the Lagrange coefficients L_m (Eq. 43), the derivative samples
 *   L'(z_p) by a type-2 NUFFT (Eq. 16), and the node weights
 *   w_p = h(-P t_p + j P a) / (L'(z_p) z_p) (Eqs. 17, 23, 27, 40).
 *   The shift a and the oversampling eta follow Sec. V (Eq. 49) from `tol`.
 * N      number of nodes (= number of coefficients), 1 <= N <= 2^28.
 * x      N nodes in radians (float64), device or host.  Not retained, but
 *        with NUFFT_DEFER_CHECK a device or pinned host array must not change
 *        before nufft_plan_check returns (its copy or its first use may still
 *        be queued).
 * tol    target relative L2 error: NUFFT_FP64 accepts [1e-12, 1e-1],
 *        NUFFT_FP32 accepts [1e-6, 1e-1]; tighter values return
 *        NUFFT_ERR_ACCURACY, non-finite or <= 0 values NUFFT_ERR_ARG.
 * prec   NUFFT_FP32 or NUFFT_FP64, optionally | NUFFT_REFINE,
 *        | NUFFT_DEFER_CHECK and | NUFFT_TOEPLITZ.
 * plan   receives the plan; owned by the caller, release with nufft_destroy.
 * The call synchronises `stream` once to check for coincident nodes: two
 * nodes whose turns t differ by less than 2^-44 modulo 1 make the systems of
 * Eqs. 47/48 numerically singular and return NUFFT_ERR_DUP_NODES (no plan).
 * A plan depends on its nodes alone, not on transforms of other plans in
 * flight, and transforms only read their plan: calls with one plan may run
 * on several streams at once.  A plan's kernels are short and latency-bound,
 * so a sequence of (plan, transforms) steps runs fastest pipelined: plan step
 * i+1 with NUFFT_DEFER_CHECK on a stream of higher priority while the
 * transforms of step i run on other streams (each waiting for an event
 * recorded after the plan call before it transforms with that plan; the FFT
 * passes hand out their tiles by counters, so concurrent transforms share
 * the SMs).  On GB300, N = 65536 with 64 right-hand sides of each kind: 0.51
 * ms per step one call after another, 0.40 with the next plan pipelined, 0.35
 * with the type-5 and type-4 inverses also on two streams; results bit for
 * bit the same.  Destroy a plan only once its creation stream has waited for
 * its transforms (see nufft_destroy).
 */
nufft_status nufft_plan(int64_t N, const double* x, double tol, int prec, nufft_stream_t stream,
                        nufft_plan_t* plan);

/*
 * nufft_plan_ex -- nufft_plan with the method's parameters set explicitly
 * (Sec. V) instead of derived from `tol`: used to study the error against the
 * attenuation mu of Eq. 49, mu = e^{-2 pi (eta N - 1) a} / (eta N - 1) with
 * gamma = e^{2 pi N a}, and to trade accuracy for plan time.  A field <= 0
 * keeps the value nufft_plan would choose for (tol, prec); `params` may be
 * NULL.  Out-of-range fields return NUFFT_ERR_ARG.  The accuracy then follows
 * from the parameters, not from `tol`, which still selects the defaults.
 */
typedef struct {
    double gamma;  /* damping gamma = rho^{-N} = e^{2 pi N a}, in (1, 1e12] */
    int eta;       /* oversampling of the log-kernel spectrum, R = eta N (Eqs. 41, 42), in [1, 64] */
    int w_plan;    /* spreading width of the plan's float64 NUFFTs (even, 4..16) */
    int w_solve;   /* spreading width of the transforms (even, 4..16) */
} nufft_params_t;

nufft_status nufft_plan_ex(int64_t N, const double* x, double tol, int prec, const nufft_params_t* params,
                           nufft_stream_t stream, nufft_plan_t* plan);

/*
 * nufft_plan_tune -- choose (gamma, eta, plan width) for these nodes, `tol`
 * and precision on this GPU (Sec. V leaves the choice open; on GB300 the
 * float64 plan's cost grows with eta).  Candidates: for each gamma in a fixed
 * set (float32 path: 30 .. 3000, plan widths 10 and 12; float64 path: 100 ..
 * 1e4) the smallest eta with the truncation error 0.4 gamma^-eta below tol/10.
 * Each candidate is accepted if the round trips c -> type-2 -> inv5 and
 * c -> type-1 -> inv4 on `batch` test vectors return c within tol/2, and
 * timed (plan + inv5 + inv4 of `batch` vectors, best of 3); the fastest
 * accepted set is written to *best (its time to *best_ms when not NULL) and
 * cached: later nufft_plan calls with the same (N, prec, tol) use it.
 * prec is NUFFT_FP32 or NUFFT_FP64 (no flags); 1 <= batch <= 1024.
 * Synchronises `stream`.  NUFFT_ERR_ACCURACY if no candidate met tol.
 */
nufft_status nufft_plan_tune(int64_t N, const double* x, double tol, int prec, int64_t batch, nufft_stream_t stream,
                             nufft_params_t* best, double* best_ms);

/*
 * nufft_inv5 -- type-5 NUFFT (Eq. 48): given samples s(t_p) of
 *   s(t) = sum_{m<N} S_m e^{j 2 pi m t}, return S.  Method of Sec. III,
 *   Fig. 1 (lower half): a_p = s(t_p) w_p (Eq. 27), type-1 NUFFT,
 *   scaling by e^{-2 pi k a} and length-N inverse DFT (Eq. 37), product with
 *   K_q (Eq. 30), length-N DFT and scaling by e^{2 pi m a} / N (Eq. 31).
 * f      batch x N samples at the plan's nodes (node order as given to nufft_plan).
 * c      batch x N coefficients S_0 .. S_{N-1}.
 * With device buffers, nufft_inv5 and nufft_inv4 can be captured in a CUDA
 * graph once a first call outside the capture has done the per-process
 * set-up; replays on new data in the same buffers give the results of
 * direct calls (the scratch then comes from the graph's own allocations).
 */
nufft_status nufft_inv5(nufft_plan_t plan, const void* f, void* c, int64_t batch, nufft_stream_t stream);

/*
 * nufft_inv5_noalloc -- the type-5 inverse of nufft_inv5 without any device
 *   allocation during the call.  The paper has no counterpart: this is for
 *   callers that cannot allocate device memory while they transform (real-time
 *   loops and embedded runtimes that forbid allocation after set-up, or
 *   processes whose device memory is handed out by an external allocator
 *   under a fixed budget).  The plan is still made by nufft_plan at set-up.
 *   Scratch is a fixed 8 MiB array inside the library image, present on
 *   every GPU that loads the library until the process exits; right-hand
 *   sides are processed one at a time through it.
 * Refined plans (NUFFT_REFINE) get the refinement of Sec. V as in
 *   nufft_inv5, also inside the static array: the float64 forward transform
 *   of the first solution, the residual and the correction take extra room.
 * Limits.  A plan whose scratch per right-hand side exceeds 8 MiB is rejected
 *   with NUFFT_ERR_ARG.  Power-of-two N that fit: up to 131072 in NUFFT_FP32
 *   and up to 65536 in NUFFT_FP64; with NUFFT_REFINE up to 65536 in
 *   NUFFT_FP32 and up to 32768 in NUFFT_FP64.  f and c must be device
 *   buffers (host buffers would need staging memory): NUFFT_ERR_ARG otherwise.
 * Set-up.  The first call on each device resolves the scratch array's
 *   device address (cudaGetSymbolAddress) with that device current; make
 *   that first call before any stream capture.
 * Concurrency.  All calls share the one scratch array, which keeps what the
 *   last call left in it.  Nothing in it needs to start at zero: every stage
 *   overwrites what it later reads, and the one stage that relies on zeros
 *   (the zero-padded grid of NUFFT_TOEPLITZ plans) clears them itself.  Calls
 *   whose work overlaps on the GPU (other streams, other threads) race on the
 *   array: order them on one stream or serialise them.
 * Arguments, layout and results as for nufft_inv5.
 */
nufft_status nufft_inv5_noalloc(nufft_plan_t plan, const void* f, void* c, int64_t batch, nufft_stream_t stream);

/*
 * nufft_inv4 -- type-4 NUFFT (Eq. 47): given A(k) = sum_p a_p e^{-j 2 pi k t_p},
 *   k = 0..N-1, return a.  Method of Sec. IV, Fig. 2: Eq. 37 on A, product
 *   with K_q (Eq. 30), Eq. 31, type-2 NUFFT at the nodes, times w_p (Eq. 40).
 * A      batch x N spectral samples.
 * a      batch x N node amplitudes (node order as given to nufft_plan).
 */
nufft_status nufft_inv4(nufft_plan_t plan, const void* A, void* a, int64_t batch, nufft_stream_t stream);

/*
 * nufft_fwd1 -- type-1 NUFFT (Eq. 32): A_k = sum_p a_p e^{-j 2 pi k t_p},
 *   k = 0..N-1, by gridding on an oversampled grid, FFT and deconvolution
 *   (Sec. II).  a: batch x N amplitudes, A: batch x N.
 */
nufft_status nufft_fwd1(nufft_plan_t plan, const void* a, void* A, int64_t batch, nufft_stream_t stream);

/*
 * nufft_fwd2 -- type-2 NUFFT (Eq. 34): s_p = sum_{m<N} S_m e^{j 2 pi m t_p},
 *   by deconvolution, inverse FFT and interpolation (Sec. II).
 *   c: batch x N coefficients, f: batch x N samples.
 */
nufft_status nufft_fwd2(nufft_plan_t plan, const void* c, void* f, int64_t batch, nufft_stream_t stream);

/*
 * nufft_fwd2_deriv -- derivative of the type-2 sum with respect to t:
 *   s'(t_p) = sum_{m<N} (j 2 pi m) S_m e^{j 2 pi m t_p}  (d/dt of Eq. 34).
 *   Used by the node gradients of the type-4/5 inverses: with S = G^{-1} f
 *   and G_{q,m} = e^{j 2 pi m t_q} (Eq. 48), dS = -G^{-1} (s' o dt).
 *   c: batch x N coefficients, f: batch x N values at the nodes.
 */
nufft_status nufft_fwd2_deriv(nufft_plan_t plan, const void* c, void* f, int64_t batch, nufft_stream_t stream);

/*
 * Node gradients of the inverses (for reverse-mode differentiation; the
 * paper has no counterpart, the formulas follow from Eqs. 47 and 48).
 * With G_{q,m} = e^{j 2 pi m t_q} and a real loss L whose gradient with
 * respect to the output is g (convention dL = Re<g, d out>):
 *   type-5, S = G^{-1} f:   u = G^{-H} g (= nufft_inv4 of g) is the gradient
 *     with respect to f, and dL/dx_q = -(1/2pi) sum_b Re(conj(u_q) s'_b(t_q)),
 *     s' the derivative type-2 of S (nufft_fwd2_deriv);
 *   type-4, a = G^{-H} A:   w = G^{-1} g (= nufft_inv5 of g) is the gradient
 *     with respect to A, and dL/dx_q = -(1/2pi) sum_b Re(conj(w'_b(t_q)) a_q).
 * u, S (resp. w, a): batch x N device buffers in the plan's precision; the
 * sum runs over the batch (right-hand sides sharing the nodes).
 * grad_x: N float64 device values, overwritten.  Scratch for the derivative
 * is taken from the device pool.
 */
nufft_status nufft_inv5_grad_nodes(nufft_plan_t plan, const void* u, const void* S, int64_t batch, double* grad_x,
                                   nufft_stream_t stream);
nufft_status nufft_inv4_grad_nodes(nufft_plan_t plan, const void* w, const void* a, int64_t batch, double* grad_x,
                                   nufft_stream_t stream);

/* nufft_destroy -- release a plan (NULL is accepted).  Its device memory is
 * returned in stream order on the plan's creation stream, so work already
 * queued there completes first; work queued on other streams must be
 * complete (or ordered before that stream) when the plan is destroyed. */
nufft_status nufft_destroy(nufft_plan_t plan);

/*
 * Batched inverses of many independent instances of uneven size in one
 * persistent kernel launch (the paper has no counterpart: each instance is
 * the method of Secs. III/IV, Figs. 1 and 2).  Each instance has its own
 * nodes, size N (2 <= N <= 16384) and kind; data are complex64 and the
 * node-dependent part is computed to float64 accuracy as in NUFFT_FP32 plans.
 * The method's parameters follow tol (Sec. V): gamma = 60, the smallest eta
 * (at most 4) whose truncation 0.4 gamma^-eta is below tol/10, spreading
 * widths 14 (plan; 12 for tol >= 1e-4) and 8 (transforms; 6 for tol >= 1e-3);
 * at tol 1e-5 that is eta = 4 (relative L2 error ~1e-6 on well-conditioned
 * nodes).  nufft_batch_tune may replace them by a faster set it validated.
 * The whole pipeline (plan and inverse) runs on every nufft_batch_run, so new
 * node values in the same buffers are picked up.
 * nufft_batch_create: `inst` is a host array of `count` descriptors of device
 *   buffers; the buffers must stay valid while the batch is used.  Allocates
 *   the descriptors, per-CTA scratch and deconvolution tables (synchronises
 *   `stream`).
 * nufft_batch_run: two memsets and one kernel launch on `stream`; capturable
 *   in a CUDA graph.
 * nufft_batch_status: per-instance status of the last run (NUFFT_OK or
 *   NUFFT_ERR_DUP_NODES), in the caller's instance order; synchronises.
 */
typedef struct {
    int64_t N;
    const double* x;   /* N nodes (radians), device */
    const void* in;    /* N complex64: samples at the nodes (kind 5) or spectrum A(k) (kind 4), device */
    void* out;         /* N complex64: coefficients (kind 5) or node amplitudes (kind 4), device */
    int kind;          /* 5 or 4 */
} nufft_instance_t;
typedef struct nufft_batch_s* nufft_batch_t;

nufft_status nufft_batch_create(int64_t count, const nufft_instance_t* inst, double tol, nufft_stream_t stream,
                                nufft_batch_t* batch);
nufft_status nufft_batch_run(nufft_batch_t batch, nufft_stream_t stream);
nufft_status nufft_batch_status(nufft_batch_t batch, int* status, nufft_stream_t stream);
/* Autotuner: runs the batch under every launch shape (1-3 CTAs per SM, 256 or
 * 512 threads, largest FFT radix 4 or 8) and keeps the fastest; then runs it
 * with candidate method parameters (gamma, eta, plan width, transforms'
 * width; Sec. V leaves the choice open) whose a-priori error fits tol --
 * truncation 0.4 gamma^-eta within tol/10, the transforms' round-off
 * 0.5 gamma 2^-24 within tol/2 -- and accepts a set only if every instance's
 * result stays within tol/2 (relative L2) of the result with the tightest set
 * (gamma 60, eta 4, widths 14 and 8); the fastest accepted set is kept.  The
 * best time goes to *best_ms when not NULL; choices are cached per (count,
 * sum of N, largest N, tol) for later batches of the same shape.  Overwrites
 * the outputs; synchronises; run it before capturing. */
nufft_status nufft_batch_tune(nufft_batch_t batch, nufft_stream_t stream, double* best_ms);
/* The launch shape in use: CTAs, threads per CTA, largest FFT radix. */
nufft_status nufft_batch_config(nufft_batch_t batch, int* ctas, int* threads, int* max_radix);
/* The method's parameters in use (gamma, eta, plan width, transforms' width). */
nufft_status nufft_batch_params(nufft_batch_t batch, nufft_params_t* params);
nufft_status nufft_batch_destroy(nufft_batch_t batch);

/* Parameters a plan chose (Sec. V).  rho = e^{-2 pi a}; gamma = rho^{-N}. */
typedef struct {
    int64_t N;
    int prec;
    double tol;
    double gamma, a, rho;
    int eta;                 /* R = eta N, Eq. 41 */
    int64_t R;
    int64_t grid_solve;      /* oversampled grid of the transforms */
    int64_t grid_plan;       /* oversampled grid of the length-R type-1 NUFFT */
    int w_solve, w_plan;     /* spreading widths (grid points) */
    double beta_solve, beta_plan;
    int64_t batch_chunk;     /* right-hand sides processed per pass */
} nufft_plan_info_t;

nufft_status nufft_plan_info(nufft_plan_t plan, nufft_plan_info_t* info);

/* Right-hand sides processed per pass of the transforms (default: set by
 * nufft_plan from the device's L2 size and the per-vector scratch). */
nufft_status nufft_plan_set_batch_chunk(nufft_plan_t plan, int64_t chunk);

/*
 * nufft_plan_export -- copy a node-dependent quantity of the plan, as N
 * complex128 values, into dst (device or host):
 *   which = 0: K_q = L(e^{j 2 pi (q/N + j a)}), q = 0..N-1      (Eqs. 10, 29)
 *   which = 1: L'(z_p), p in node order                        (Sec. III-D)
 *   which = 2: w_p = h(-N t_p + j N a) / (L'(z_p) z_p)          (Eqs. 27, 40)
 * Synchronises `stream`.
 */
nufft_status nufft_plan_export(nufft_plan_t plan, int which, void* dst, nufft_stream_t stream);

/*
 * nufft_plan_save / nufft_plan_restore -- no counterpart in the paper.  For
 * reverse-mode differentiation, which needs the plan again in the backward
 * pass: keep the two node-dependent quantities that cost the plan its FFTs,
 * K_q = L(e^{j 2 pi (q/N + j a)}) (Eqs. 10, 29) and L'(z_p) (Sec. III-D), 32
 * bytes per node, instead of the whole plan, and recompute the rest.
 * nufft_plan_save copies them, as N complex128 values each (K in q order,
 *   D in node order), into the device buffers K and D, asynchronously on
 *   `stream`.  NUFFT_ERR_ARG for null or host pointers.
 * nufft_plan_restore makes a plan for the nodes x from them: arguments as for
 *   nufft_plan_ex, which must be those of the saved plan (same node values,
 *   N, tol, precision and method parameters; pass the saved plan's gamma,
 *   eta and widths from nufft_plan_info to be independent of the tuner's
 *   cache), plus the saved K and D (device, read in stream order: they must
 *   stay valid until the call's work on `stream` has run).  Only the node
 *   geometry (exact turns, cell sort, extended node list, coincident-node
 *   check), the node phases and the weights w_p of Eqs. 27/40 are computed;
 *   the log-kernel type-1, the FFTs and the type-2 of the plan are skipped.
 *   NUFFT_REFINE and NUFFT_DEFER_CHECK are accepted; NUFFT_TOEPLITZ is not
 *   (NUFFT_ERR_ARG).  Results are those of the saved plan.
 */
nufft_status nufft_plan_save(nufft_plan_t plan, void* K, void* D, nufft_stream_t stream);
nufft_status nufft_plan_restore(int64_t N, const double* x, double tol, int prec, const nufft_params_t* params,
                                const void* K, const void* D, nufft_stream_t stream, nufft_plan_t* plan);

/*
 * nufft_plan_check -- no counterpart in the paper.  Waits for the plan's
 * kernels on its stream and returns NUFFT_ERR_DUP_NODES if two nodes coincide
 * modulo 2 pi (the inverse does not exist; results of the plan are not to be
 * used), else NUFFT_OK.  For plans made with NUFFT_DEFER_CHECK this is where
 * that condition surfaces; for the others nufft_plan already reported it.
 */
nufft_status nufft_plan_check(nufft_plan_t plan);

/*
 * nufft_stream_check -- no counterpart in the paper.  Synchronises `stream`
 * and the library's copy streams of the current device (so pinned host
 * outputs are complete) and reports whether a bounded wait inside one of the library's kernels on
 * the current device gave up since the last call: the TMA-fed FFT passes wait
 * on shared-memory barriers for their input tiles with an iteration limit,
 * and on expiry count the event, let their copies land and return without
 * writing that tile.  Returns NUFFT_ERR_TIMEOUT (and clears the count) if
 * that happened, NUFFT_ERR_CUDA on a CUDA error, else NUFFT_OK.  Results of
 * the calls in between are then not to be trusted.
 */
nufft_status nufft_stream_check(nufft_stream_t stream);

/* Drop the cache of node-independent tables (deconvolution and scaling
 * factors, FFT twiddles) kept per (N, precision, tolerance, parameters) and
 * the parameter sets nufft_plan_tune chose.  Plans that are alive keep their
 * own reference. */
nufft_status nufft_cache_clear(void);

/*
 * Tracing (no counterpart in the paper; for measurement).  Every kernel the
 * library launches is counted.  While tracing is enabled, each launch is
 * bracketed by CUDA events recorded on its own stream and attributed to a
 * kernel class ("fft_pass", "spread", "interp", "select", "place",
 * "pointwise", "geometry", "plan_table", "plan_stage", "bluestein"; float64
 * launches of a class are reported as "<class>_f64") together with its
 * algorithmic byte count (the bytes the kernel must read and write
 * once).  nufft_profile_enable(1) clears earlier records.
 * nufft_profile_read synchronises the recorded events and returns one entry
 * per class that launched, at most `cap`, in `out`.
 */
typedef struct {
    char name[32];
    int64_t launches;
    double ms;        /* summed event time of the launches */
    double bytes;     /* summed algorithmic bytes */
} nufft_profile_entry_t;

nufft_status nufft_profile_enable(int on);
nufft_status nufft_profile_read(nufft_profile_entry_t* out, int cap, int* count);
int64_t nufft_launch_count(void);

/*
 * Measurement utility (no counterpart in the paper): the device's sustained
 * fused multiply-add rate in float32 (prec = NUFFT_FP32) or float64
 * (NUFFT_FP64), from a kernel of independent FMA chains filling every SM,
 * timed with CUDA events on `stream` after a warm-up launch.  Writes
 * TFLOP/s (2 flops per FMA) to *tflops; synchronises the stream.  It is the
 * denominator for kernels bound by arithmetic rather than memory (the plan's
 * float64 stages).  NUFFT_ERR_ARG for a null pointer or another precision.
 */
nufft_status nufft_measure_fma(int prec, double* tflops, nufft_stream_t stream);

const char* nufft_status_string(nufft_status st);
const char* nufft_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* NUFFT45_H */

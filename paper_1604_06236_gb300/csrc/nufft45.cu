// Host runtime and C ABI of the nufft45 library: parameter choice (Sec. V),
// the cache of node-independent tables, the node-dependent plan (Sec. III,
// Fig. 1 upper half), and the type-1/2/4/5 transforms (Figs. 1 and 2).
#include "internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

namespace nufft45 {

// --------------------------------------------------------------- errors ----
static thread_local char g_msg[512] = "";

nufft_status fail(nufft_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

nufft_status cuda_fail(cudaError_t e, const char* expr, const char* file, int line) {
    const nufft_status st = (e == cudaErrorMemoryAllocation) ? NUFFT_ERR_ALLOC : NUFFT_ERR_CUDA;
    fail(st, "%s failed: %s (%s:%d)", expr, cudaGetErrorString(e), file, line);
    cudaGetLastError();   // clear a sticky launch error so the context stays usable
    return st;
}

// Test hook: make the next `count` device allocations of this library fail
// as if the device were out of memory.
static int g_fail_allocs = 0;

// ------------------------------------------------- stream-ordered arenas ---
struct Arena {
    char* base = nullptr;
    size_t cap = 0, used = 0;
    cudaStream_t stream = nullptr;
    nufft_status reserve(size_t bytes, cudaStream_t s) {
        stream = s;
        cap = bytes;
        if (g_fail_allocs > 0) { --g_fail_allocs; return fail(NUFFT_ERR_ALLOC, "injected allocation failure"); }
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), bytes, s);
        if (e != cudaSuccess) { base = nullptr; return cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__); }
        return NUFFT_OK;
    }
    template <typename X> X* take(size_t count) {
        size_t off = (used + 255) & ~(size_t)255;
        used = off + count * sizeof(X);
        return reinterpret_cast<X*>(base + off);
    }
    void release() {
        if (base) cudaFreeAsync(base, stream);
        base = nullptr;
    }
    // free in the order of another stream (one that has waited for every use)
    void release_on(cudaStream_t s) {
        stream = s;
        release();
    }
};

// a size accumulator with the same alignment rule as Arena::take
struct Sizer {
    size_t used = 0;
    template <typename X> void add(size_t count) { used = ((used + 255) & ~(size_t)255) + count * sizeof(X); }
};

static void init_pool_once() {
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;   // keep freed blocks for reuse instead of returning them
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

// -------------------------------------------------------- parameters -------
struct Params {
    int64_t N = 0;
    int prec = 0;
    double tol = 0;
    double gamma = 0, a = 0, rho = 0, log_rho = 0, rhoP = 0;
    int eta = 0;
    int64_t R = 0;
    int64_t ns = 0;
    int64_t K0s = 0, K0R = 0;
    KernelShape ks_solve{0, 0}, ks_plan{0, 0};
    bool refine = false;   // one refinement step per inverse (Sec. V)
    bool toeplitz = false; // middle stage as a linear convolution with L (no rho^-m scaling)
    int halo = 0;          // halo width of the transforms' extended node list
};

// oversampled grid length >= m: a power of two when that costs at most 30%
// more points (the power-of-two FFT passes are the fastest), otherwise the
// smallest 2,3,5,7-smooth length
static int64_t grid_size(int64_t m) {
    int64_t p2 = 1;
    while (p2 < m) p2 <<= 1;
    const int64_t sm = next_smooth(m);
    return (double)p2 <= 1.3 * (double)sm ? p2 : sm;
}

// ES kernel shape for an even width w on an oversampling-2 grid
static KernelShape es_shape(int w) { return KernelShape{w, 2.30 * w}; }

// Sec. V: the truncation of Eq. 42 at R = eta P leaves a relative error close
// to mu ~ gamma^-eta (Eq. 49 with gamma = e^{2 pi P a}); round-off in the
// scaling by e^{2 pi p a} of Eqs. 31 and 43 grows with gamma.  float64:
// gamma = 1000 and eta from tol; float32 transforms: gamma = 100, eta = 3 and
// plan width 12, which leave the float64 plan accurate to ~1e-7 (truncation
// 0.4 gamma^-eta ~ 4e-7, kernel error ~1e-11) while the float32 stages bring
// ~2e-6; the plan's float64 work is what these choices keep small.
static nufft_status choose_params(int64_t N, double tol, int prec, Params& p) {
    p.N = N;
    p.prec = prec;
    p.tol = tol;
    int w_solve, w_plan;
    if (prec == NUFFT_FP64) {
        if (tol < 1e-12) return fail(NUFFT_ERR_ACCURACY, "tol %g below what the float64 path attains (1e-12)", tol);
        p.gamma = 1000.0;
        p.eta = std::max(2, (int)std::ceil(std::log10(4.0 / tol) / 3.0));
        w_plan = w_solve = tol < 1e-8 ? 16 : 12;
    } else {
        if (tol < 1e-6) return fail(NUFFT_ERR_ACCURACY, "tol %g below what the float32 path attains (1e-6)", tol);
        p.gamma = 100.0;
        p.eta = 3;
        w_plan = 12;
        w_solve = 8;
    }
    p.ks_solve = es_shape(w_solve);
    p.ks_plan = es_shape(w_plan);
    return NUFFT_OK;
}

// explicit parameters (fields <= 0 keep the defaults), then the derived quantities
static nufft_status apply_params(const nufft_params_t* q, Params& p) {
    if (q) {
        if (q->gamma > 0) {
            if (!(q->gamma > 1.0) || !std::isfinite(q->gamma) || q->gamma > 1e12)
                return fail(NUFFT_ERR_ARG, "gamma %g out of range (1, 1e12]", q->gamma);
            p.gamma = q->gamma;
        }
        if (q->eta > 0) {
            if (q->eta > 64) return fail(NUFFT_ERR_ARG, "eta %d out of range [1, 64]", q->eta);
            p.eta = q->eta;
        }
        for (int w : {q->w_plan, q->w_solve})
            if (w > 0 && (w < 4 || w > 16 || (w & 1)))
                return fail(NUFFT_ERR_ARG, "spreading width %d is not an even number in [4, 16]", w);
        if (q->w_plan > 0) p.ks_plan = es_shape(q->w_plan);
        if (q->w_solve > 0) p.ks_solve = es_shape(q->w_solve);
    }
    const int64_t N = p.N;
    p.log_rho = -std::log(p.gamma) / (double)N;
    p.a = std::log(p.gamma) / (2.0 * M_PI * (double)N);
    p.rho = std::exp(p.log_rho);
    p.rhoP = 1.0 / p.gamma;
    p.R = (int64_t)p.eta * N;
    const int wmax = std::max(p.ks_solve.w, p.ks_plan.w);
    p.ns = grid_size(std::max<int64_t>(2 * N, 2 * wmax));
    p.K0s = N / 2;
    p.K0R = p.R / 2;
    p.halo = wmax;   // the plan's float64 transforms (width w_plan) share the transforms' node list
    return NUFFT_OK;
}

// ------------------------------------------ node-independent tables --------
struct Tables {
    Params prm;
    FFTPlan fft_ns, fft_P;          // solve precision
    FFTPlan fft_ns64, fft_P64;      // float64-accuracy transforms in double-float arithmetic
    // float64 plan tables
    double* fold = nullptr;         // Lambda_k / phihat((k mod P) - K0), k < R
    double* plan_place = nullptr;   // 1/phihat (plan width, grid ns), k < P
    double* sneg64 = nullptr;       // rho^-k / P
    // solve tables, solve precision
    void* fac1 = nullptr;           // 1/phihat
    void* fac5 = nullptr;           // rho^k/phihat
    void* fac4 = nullptr;           // rho^-k/(P phihat)
    void* rpos = nullptr;           // rho^k
    void* sneg = nullptr;           // rho^-k/P
    void* mem = nullptr;
    ~Tables() { cudaFree(mem); }
};

using TablesPtr = std::shared_ptr<Tables>;
static std::mutex g_cache_mu;
static std::map<std::tuple<int64_t, int, double, double, int, int, int>, TablesPtr> g_cache;
// parameters nufft_plan_tune chose, per (N, precision, tol); nufft_plan uses them
static std::map<std::tuple<int64_t, int, double>, nufft_params_t> g_tuned;

static nufft_status make_tables(const Params& prm, cudaStream_t s, TablesPtr& out) {
    TablesPtr t = std::make_shared<Tables>();
    t->prm = prm;
    const int64_t P = prm.N;
    const size_t es = prm.prec == NUFFT_FP64 ? sizeof(double) : sizeof(float);
    Sizer z;
    z.add<double>(prm.R); z.add<double>(P); z.add<double>(P);
    for (int i = 0; i < 5; ++i) z.add<char>(es * P);
    if (g_fail_allocs > 0) { --g_fail_allocs; return fail(NUFFT_ERR_ALLOC, "injected allocation failure"); }
    NUFFT_CUDA_TRY(cudaMalloc(&t->mem, z.used));
    Arena ar;
    ar.base = (char*)t->mem;
    ar.cap = z.used;
    t->fold = ar.take<double>(prm.R);
    t->plan_place = ar.take<double>(P);
    t->sneg64 = ar.take<double>(P);
    t->fac1 = ar.take<char>(es * P);
    t->fac5 = ar.take<char>(es * P);
    t->fac4 = ar.take<char>(es * P);
    t->rpos = ar.take<char>(es * P);
    t->sneg = ar.take<char>(es * P);
    nufft_status st;
    const int sp = prm.prec == NUFFT_FP64 ? 2 : 1;
    if ((st = fft_make(t->fft_ns, prm.ns, sp, s)) != NUFFT_OK) return st;
    if ((st = fft_make(t->fft_P, P, sp, s)) != NUFFT_OK) return st;
    // the plan's float64-accuracy FFTs run in double-float arithmetic: GB300
    // issues float32 at 64x its float64 rate
    if ((st = fft_make(t->fft_ns64, prm.ns, 3, s)) != NUFFT_OK) return st;
    if ((st = fft_make(t->fft_P64, P, 3, s)) != NUFFT_OK) return st;
    GLRule glR, glS;
    gauss_legendre_half(2 + (3 * prm.ks_plan.w) / 2 + 4, glR);
    gauss_legendre_half(2 + (3 * prm.ks_solve.w) / 2 + 4, glS);
    launch_table(prm.ks_plan, glR, prm.ns, prm.K0s, prm.R, prm.log_rho, 6, P, t->fold, nullptr, s);
    launch_table(prm.ks_plan, glR, prm.ns, prm.K0s, P, prm.log_rho, 0, P, t->plan_place, nullptr, s);
    launch_table(prm.ks_plan, glR, prm.ns, prm.K0s, P, prm.log_rho, 5, P, t->sneg64, nullptr, s);
    const bool d = prm.prec == NUFFT_FP64;
    void* tabs[5] = {t->fac1, t->fac5, t->fac4, t->rpos, t->sneg};
    const int modes[5] = {0, 1, 2, 4, 5};
    for (int i = 0; i < 5; ++i)
        launch_table(prm.ks_solve, glS, prm.ns, prm.K0s, P, prm.log_rho, modes[i], P,
                     d ? (double*)tabs[i] : nullptr, d ? nullptr : (float*)tabs[i], s);
    NUFFT_CUDA_TRY(cudaGetLastError());
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    out = t;
    return NUFFT_OK;
}

static nufft_status get_tables(const Params& prm, cudaStream_t s, TablesPtr& out) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto key = std::make_tuple(prm.N, prm.prec, prm.tol, prm.gamma, prm.eta, prm.ks_plan.w, prm.ks_solve.w);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) { out = it->second; return NUFFT_OK; }
    nufft_status st = make_tables(prm, s, out);
    if (st == NUFFT_OK) g_cache[key] = out;
    return st;
}

}  // namespace nufft45

using namespace nufft45;

// ------------------------------------------------------------------ plan ---
// one FFT as one traced unit: its passes run back to back on the stream
template <typename Fn, typename... A>
nufft_status traced_fft(cudaStream_t s, bool f64, Fn&& fn, A&&... a) {
    LaunchGroup g(s, K_FFT, f64);
    return fn(std::forward<A>(a)...);
}

struct nufft_plan_s {
    Params prm;
    TablesPtr tab;
    cudaStream_t stream = nullptr;
    Arena mem;                       // node-dependent buffers
    Geometry gs;
    uint64_t* T = nullptr;
    double2* K64 = nullptr;
    double2* D64 = nullptr;
    double2* w64 = nullptr;
    void* Ks = nullptr;              // K in the solve precision
    void* wt1_ext = nullptr;         // e^{-j 2 pi K0 t}, extended slot order
    void* wt5_ext = nullptr;         // w e^{-j 2 pi K0 t}
    void* wt2_srt = nullptr;         // e^{+j 2 pi K0 t}, sorted slot order
    void* wt4_srt = nullptr;         // w e^{+j 2 pi K0 t}
    double2* modm64_ext = nullptr;   // float64 e^{-j 2 pi K0 t}, extended slot order
    double2* modp64_srt = nullptr;   // float64 e^{+j 2 pi K0 t}, sorted slot order
    int64_t chunk = 1;
    void* FL = nullptr;              // DFT of L_0..L_P zero-padded to ns, / ns (solve precision; toeplitz)
    int* dup_host = nullptr;         // pinned copy of the duplicate-node flag
    cudaEvent_t dup_ev = nullptr;    // recorded after that copy
};

namespace {

// Pinned host words for the duplicate-node flags: a plan's flag is copied
// back asynchronously, so nufft_plan_check waits for the plan's own kernels
// only, not for work queued after them.  A word returns to the pool once its
// copy has landed.
struct PinnedWords {
    std::mutex mu;
    std::vector<int*> free_;
    std::vector<std::pair<int*, cudaEvent_t>> pending;   // released, copy maybe in flight
    int* acquire() {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = 0; i < pending.size();) {
            if (cudaEventQuery(pending[i].second) != cudaErrorNotReady) {
                cudaGetLastError();
                cudaEventDestroy(pending[i].second);
                free_.push_back(pending[i].first);
                pending[i] = pending.back();
                pending.pop_back();
            } else {
                ++i;
            }
        }
        if (free_.empty()) {
            int* block = nullptr;
            if (cudaHostAlloc(reinterpret_cast<void**>(&block), 1024 * sizeof(int), cudaHostAllocPortable) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            for (int i = 0; i < 1024; ++i) free_.push_back(block + i);
        }
        int* w = free_.back();
        free_.pop_back();
        return w;
    }
    void release(int* w, cudaEvent_t ev) {
        std::lock_guard<std::mutex> lk(mu);
        if (ev) pending.emplace_back(w, ev);
        else free_.push_back(w);
    }
};
PinnedWords& pinned_words() {
    static PinnedWords* p = new PinnedWords();   // outlives static destruction order
    return *p;
}

}  // namespace

namespace {

enum MemLoc { LOC_DEVICE, LOC_PINNED, LOC_PAGEABLE };

MemLoc mem_loc(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return LOC_PAGEABLE; }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return LOC_DEVICE;
    return at.type == cudaMemoryTypeHost ? LOC_PINNED : LOC_PAGEABLE;
}

bool is_device_ptr(const void* p) { return mem_loc(p) == LOC_DEVICE; }

// per-device streams for host <-> device copies of pinned buffers, so that
// they overlap the transforms queued on the caller's stream
struct CopyStreams { cudaStream_t h2d = nullptr, d2h = nullptr; };
nufft_status copy_streams(CopyStreams& out) {
    static std::mutex mu;
    static CopyStreams per_dev[64];
    int dev = 0;
    NUFFT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(NUFFT_ERR_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    CopyStreams& c = per_dev[dev];
    if (!c.h2d) NUFFT_CUDA_TRY(cudaStreamCreateWithFlags(&c.h2d, cudaStreamNonBlocking));
    if (!c.d2h) NUFFT_CUDA_TRY(cudaStreamCreateWithFlags(&c.d2h, cudaStreamNonBlocking));
    out = c;
    return NUFFT_OK;
}

// make `waiter` wait for the work queued so far on `on`
nufft_status order_after(cudaStream_t waiter, cudaStream_t on) {
    cudaEvent_t e = nullptr;
    NUFFT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t r = cudaEventRecord(e, on);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(waiter, e, 0);
    cudaEventDestroy(e);   // released once the recorded work completes
    if (r != cudaSuccess) return cuda_fail(r, "stream ordering", __FILE__, __LINE__);
    return NUFFT_OK;
}

size_t solve_elem(const Params& p) { return p.prec == NUFFT_FP64 ? sizeof(double2) : sizeof(float2); }

// queue the copy of the duplicate-node flag behind the plan's kernels
nufft_status plan_dup_queue(nufft_plan_s* pl) {
    pl->dup_host = pinned_words().acquire();
    if (!pl->dup_host) return fail(NUFFT_ERR_ALLOC, "pinned host word for the duplicate-node flag");
    NUFFT_CUDA_TRY(cudaEventCreateWithFlags(&pl->dup_ev, cudaEventDisableTiming));
    NUFFT_CUDA_TRY(cudaMemcpyAsync(pl->dup_host, pl->gs.dup_flag, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
    NUFFT_CUDA_TRY(cudaEventRecord(pl->dup_ev, pl->stream));
    return NUFFT_OK;
}

// wait for the plan's kernels (not for later work on its stream) and read
// the duplicate-node flag they set
nufft_status plan_dup_check(nufft_plan_s* pl) {
    if (!pl->dup_ev) return fail(NUFFT_ERR_ARG, "plan has no queued check");
    NUFFT_CUDA_TRY(cudaEventSynchronize(pl->dup_ev));
    return *pl->dup_host ? fail(NUFFT_ERR_DUP_NODES, "two nodes coincide modulo 2 pi") : NUFFT_OK;
}

void plan_dup_release(nufft_plan_s* pl) {
    if (pl->dup_host) {
        pinned_words().release(pl->dup_host, pl->dup_ev);
    } else if (pl->dup_ev) {
        cudaEventDestroy(pl->dup_ev);
    }
    pl->dup_host = nullptr;
    pl->dup_ev = nullptr;
}

int64_t per_item_elems(const nufft_plan_s* pl) {
    const Tables& t = *pl->tab;
    return pl->prm.ns + fft_work_elems(t.fft_ns) + pl->prm.N + fft_work_elems(t.fft_P);
}

// Ksv, Dsv: K_q and L'(z_p) saved from an earlier plan of the same nodes and
// parameters (nufft_plan_restore): only the geometry, the node phases and the
// weights are then computed
nufft_status run_plan(nufft_plan_s* pl, const double* x_dev, const double2* Ksv = nullptr,
                      const double2* Dsv = nullptr) {
    const Params& prm = pl->prm;
    const Tables& tab = *pl->tab;
    cudaStream_t s = pl->stream;
    const int64_t N = prm.N, P = N;
    const bool f32 = prm.prec == NUFFT_FP32;
    const size_t es = solve_elem(prm);
    // persistent buffers
    Sizer z;
    z.add<uint64_t>(N);
    z.add<int>(N); z.add<int>(N); z.add<double>(N); z.add<float>(N);
    z.add<int>(2 * N); z.add<int>(2 * N); z.add<double>(2 * N); z.add<float>(2 * N);
    z.add<int>(prm.ns + prm.halo + 1); z.add<int>(1);
    z.add<double2>(P); z.add<double2>(N); z.add<double2>(N);
    z.add<char>(es * P);
    z.add<char>(es * 2 * N); z.add<char>(es * 2 * N); z.add<char>(es * N); z.add<char>(es * N);
    z.add<double2>(2 * N); z.add<double2>(N);
    if (prm.toeplitz) z.add<char>(es * prm.ns);
    nufft_status st = pl->mem.reserve(z.used, s);
    if (st != NUFFT_OK) return st;
    Arena& m = pl->mem;
    pl->T = m.take<uint64_t>(N);
    Geometry& gs = pl->gs;
    gs.srt_perm = m.take<int>(N); gs.srt_cell = m.take<int>(N); gs.srt_frac = m.take<double>(N);
    gs.srt_fracf = m.take<float>(N);
    gs.ext_perm = m.take<int>(2 * N); gs.ext_cell = m.take<int>(2 * N); gs.ext_frac = m.take<double>(2 * N);
    gs.ext_fracf = m.take<float>(2 * N);
    gs.cstart = m.take<int>(prm.ns + prm.halo + 1);
    gs.dup_flag = m.take<int>(1);
    pl->K64 = m.take<double2>(P);
    pl->D64 = m.take<double2>(N);
    pl->w64 = m.take<double2>(N);
    pl->Ks = m.take<char>(es * P);
    pl->wt1_ext = m.take<char>(es * 2 * N);
    pl->wt5_ext = m.take<char>(es * 2 * N);
    pl->wt2_srt = m.take<char>(es * N);
    pl->wt4_srt = m.take<char>(es * N);
    pl->modm64_ext = m.take<double2>(2 * N);
    pl->modp64_srt = m.take<double2>(N);
    if (prm.toeplitz) pl->FL = m.take<char>(es * prm.ns);

    if (Ksv) {
        // restored plan: the saved K_q and L'(z_p), then the per-node work
        Sizer zr;
        const int64_t geo_ints = geometry_scratch_ints(N, prm.ns);
        zr.add<int>(geo_ints);
        zr.add<double2>((size_t)N);
        zr.add<unsigned long long>(1);
        Arena tmp;
        if ((st = tmp.reserve(zr.used, s)) != NUFFT_OK) return st;
        int* geo = tmp.take<int>(geo_ints);
        double2* beta64 = tmp.take<double2>((size_t)N);
        unsigned long long* sumT = tmp.take<unsigned long long>(1);
        if ((st = build_geometry(gs, x_dev, pl->T, N, prm.ns, prm.halo, f32, geo, sumT, s)) != NUFFT_OK) {
            tmp.release();
            return st;
        }
        launch_node_phases(pl->T, gs, (uint64_t)prm.K0s, (uint64_t)P, 0, pl->modm64_ext, pl->modp64_srt, beta64,
                           nullptr, s);
        NUFFT_CUDA_TRY(cudaMemcpyAsync(pl->K64, Ksv, sizeof(double2) * P, cudaMemcpyDeviceToDevice, s));
        NUFFT_CUDA_TRY(cudaMemcpyAsync(pl->D64, Dsv, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s));
        if (f32) launch_to_solve<float>(pl->K64, P, 1.0, (float2*)pl->Ks, s);
        else NUFFT_CUDA_TRY(cudaMemcpyAsync(pl->Ks, Ksv, sizeof(double2) * P, cudaMemcpyDeviceToDevice, s));
        if (f32) {
            launch_weights<float>(pl->T, gs, pl->D64, pl->modp64_srt, beta64, prm.rhoP, pl->w64,
                                  (float2*)pl->wt2_srt, (float2*)pl->wt4_srt, (float2*)pl->wt1_ext,
                                  (float2*)pl->wt5_ext, s);
        } else {
            launch_weights<double>(pl->T, gs, pl->D64, pl->modp64_srt, beta64, prm.rhoP, pl->w64,
                                   (double2*)pl->wt2_srt, (double2*)pl->wt4_srt, (double2*)pl->wt1_ext,
                                   (double2*)pl->wt5_ext, s);
        }
        NUFFT_CUDA_TRY(cudaGetLastError());
        tmp.release();
        return NUFFT_OK;
    }

    // temporaries of the plan
    const int eta = prm.eta;
    Sizer zt;
    const int64_t geo_ints = geometry_scratch_ints(N, prm.ns);
    zt.add<int>(geo_ints);
    zt.add<double2>((size_t)N);                                          // e^{-j 2 pi P t_p}
    zt.add<double2>((size_t)eta * 2 * N);                                // strengths per extended slot (dd)
    zt.add<double2>((size_t)eta * prm.ns);                               // grids
    zt.add<double2>((size_t)eta * fft_work_elems(tab.fft_ns64));
    zt.add<double2>(P); zt.add<double2>(fft_work_elems(tab.fft_P64));
    zt.add<unsigned long long>(1);
    zt.add<double>((size_t)N * prm.ks_plan.w);                           // kernel values

    Arena tmp;
    if ((st = tmp.reserve(zt.used, s)) != NUFFT_OK) return st;
    int* geo = tmp.take<int>(geo_ints);
    double2* beta64 = tmp.take<double2>((size_t)N);
    double2* sx = tmp.take<double2>((size_t)eta * 2 * N);
    double2* grid = tmp.take<double2>((size_t)eta * prm.ns);
    double2* gwork = tmp.take<double2>((size_t)eta * fft_work_elems(tab.fft_ns64));
    double2* vecP = tmp.take<double2>(P);
    double2* workP = tmp.take<double2>(fft_work_elems(tab.fft_P64));
    unsigned long long* sumT = tmp.take<unsigned long long>(1);
    double* ktab = tmp.take<double>((size_t)N * prm.ks_plan.w);

    // nodes: exact turns, sum t_p mod 1 for the constant phase of Eq. 29, and
    // the cell-sorted geometry on the transforms' grid (halo for the wider width)
    if ((st = build_geometry(gs, x_dev, pl->T, N, prm.ns, prm.halo, f32, geo, sumT, s)) != NUFFT_OK) {
        tmp.release();
        return st;
    }
    // v(q/P) (Eqs. 13, 19, 28): the type-1 of unit strengths at k = P r + m,
    // k < R = eta P, is the type-1 at m < P of the strengths
    // e^{-j 2 pi P r t_p}, r < eta (one spread of eta right-hand sides and a
    // batched FFT on the transforms' grid), folded by Eq. 7 with Eq. 41's
    // coefficients and the deconvolution
    // (the spread, its grid and the FFT's input stay in double-float)
    launch_node_phases(pl->T, gs, (uint64_t)prm.K0s, (uint64_t)P, eta, pl->modm64_ext, pl->modp64_srt, beta64, sx, s);
    launch_spread_plan_dd(gs, prm.ks_plan, sx, 2 * N, grid, eta, s, ktab);
    double2* B = nullptr;
    if ((st = traced_fft(s, true, fft_exec_dd, tab.fft_ns64, grid, gwork, eta, -1, s, &B, kDdIn)) != NUFFT_OK) {
        tmp.release();
        return st;
    }
    launch_fold(B, prm.ns, prm.K0s, tab.fold, P, eta, vecP, s);
    double2* v = nullptr;
    if ((st = traced_fft(s, true, fft_exec_dd, tab.fft_P64, vecP, workP, 1, +1, s, &v, 0)) != NUFFT_OK) { tmp.release(); return st; }
    // K_q (Eq. 29)
    // K_q (Eq. 29), with the copy that the DFT of Eq. 43 transforms in place
    launch_kernel_samples(v, P, sumT, pl->K64, f32 ? (float2*)pl->Ks : nullptr, f32 ? nullptr : (double2*)pl->Ks,
                          vecP, s);
    double2* F = nullptr;
    if ((st = traced_fft(s, true, fft_exec_dd, tab.fft_P64, vecP, workP, 1, -1, s, &F, 0)) != NUFFT_OK) { tmp.release(); return st; }
    if (prm.toeplitz) {
        // DFT of L_0..L_P zero-padded to the grid size (ns >= 2P), / ns, for
        // the middle stage as a linear convolution
        launch_lagrange_pad(F, P, prm.rhoP, tab.sneg64, prm.ns, grid, s);
        double2* FLd = nullptr;
        if ((st = traced_fft(s, true, fft_exec_dd, tab.fft_ns64, grid, gwork, 1, -1, s, &FLd, 0)) != NUFFT_OK) { tmp.release(); return st; }
        if (f32) launch_to_solve<float>(FLd, prm.ns, 1.0 / (double)prm.ns, (float2*)pl->FL, s);
        else launch_to_solve<double>(FLd, prm.ns, 1.0 / (double)prm.ns, (double2*)pl->FL, s);
    }
    // L_m (Eq. 43) and the coefficients (m+1) L_{m+1} of L' (Eq. 16) on the
    // grid, then L'(z_p) by a type-2 NUFFT on the transforms' grid (float64,
    // plan width)
    launch_lcoef_place(F, P, tab.sneg64, prm.K0s, tab.plan_place, prm.ns, grid, s);
    // (the FFT leaves its result in double-float for the interpolation)
    double2* gsp = nullptr;
    if ((st = traced_fft(s, true, fft_exec_dd, tab.fft_ns64, grid, gwork, 1, +1, s, &gsp, kDdOut)) != NUFFT_OK) {
        tmp.release();
        return st;
    }
    launch_interp_plan_dd(gs, prm.ks_plan, gsp, ktab, pl->modp64_srt, pl->D64, s);
    // w_p (Eqs. 27, 40) and the per-slot weights of the transforms, with
    // e^{-j 2 pi P t_p} (the factor of Eq. 17) from the node phases
    const double2* beta = beta64;
    if (f32) {
        launch_weights<float>(pl->T, gs, pl->D64, pl->modp64_srt, beta, prm.rhoP, pl->w64, (float2*)pl->wt2_srt,
                              (float2*)pl->wt4_srt, (float2*)pl->wt1_ext, (float2*)pl->wt5_ext, s);
    } else {
        launch_weights<double>(pl->T, gs, pl->D64, pl->modp64_srt, beta, prm.rhoP, pl->w64,
                               (double2*)pl->wt2_srt, (double2*)pl->wt4_srt, (double2*)pl->wt1_ext,
                               (double2*)pl->wt5_ext, s);
    }
    NUFFT_CUDA_TRY(cudaGetLastError());
    tmp.release();
    return NUFFT_OK;
}

// ------------------------------------------------------------ transforms ---
enum Op { OP_INV5, OP_INV4, OP_FWD1, OP_FWD2, OP_FWD2D };

template <typename T>
nufft_status run_chunk(const nufft_plan_s* pl, Op op, const c2<T>* in, c2<T>* out, int64_t bc, c2<T>* gA, c2<T>* gW,
                       c2<T>* vA, c2<T>* vW, cudaStream_t s) {
    const Params& prm = pl->prm;
    const Tables& tab = *pl->tab;
    const int64_t N = prm.N, P = N, ns = prm.ns;
    const T* fac1 = (const T*)tab.fac1;
    const T* fac5 = (const T*)tab.fac5;
    const T* fac4 = (const T*)tab.fac4;
    const T* rpos = (const T*)tab.rpos;
    const T* sneg = (const T*)tab.sneg;
    const c2<T>* K = (const c2<T>*)pl->Ks;
    nufft_status st;
    c2<T>* r = nullptr;
    // the middle stage of Eqs. 37, 30, 31 on the vector in vA (already scaled
    // by rho^k); returns the pointer holding DFT(K * P IDFT(.)) before rho^-m/P
    // float64 data goes through the double-float transforms (float pairs on the
    // float32 pipes, ~2^-48): GB300 issues float64 at 1/64 of the float32 rate
    auto fft = [&](bool grid_size, c2<T>* buf, c2<T>* work, int dir, c2<T>** res) -> nufft_status {
        LaunchGroup g(s, K_FFT, sizeof(T) == 8);
        if constexpr (sizeof(T) == 8) {
            return fft_exec_dd(grid_size ? tab.fft_ns64 : tab.fft_P64, reinterpret_cast<double2*>(buf),
                               reinterpret_cast<double2*>(work), bc, dir, s, reinterpret_cast<double2**>(res));
        } else {
            return fft_exec<T>(grid_size ? tab.fft_ns : tab.fft_P, buf, work, bc, dir, s, res);
        }
    };
    auto middle = [&](c2<T>** res) -> nufft_status {
        c2<T>* r1 = nullptr;
        nufft_status e = fft(false, vA, vW, +1, &r1);
        if (e != NUFFT_OK) return e;
        launch_pointwise<T>(r1, P, r1, P, P, K, nullptr, bc, s);
        return fft(false, r1, r1 == vA ? vW : vA, -1, res);
    };
    // grid (already placed) -> type-2 at the nodes times wt_srt: the float64
    // path keeps the FFT's result in double-float and interpolates in it
    auto grid_to_nodes = [&](const void* wt_srt) -> nufft_status {
        if constexpr (sizeof(T) == 8) {
            double2* rd = nullptr;
            nufft_status e = traced_fft(s, true, fft_exec_dd, tab.fft_ns64, reinterpret_cast<double2*>(gA),
                                        reinterpret_cast<double2*>(gW), bc, +1, s, &rd, kDdOut);
            if (e != NUFFT_OK) return e;
            launch_interp_dd(pl->gs, prm.ks_solve, rd, (const double2*)wt_srt, reinterpret_cast<double2*>(out), N,
                             bc, s);
            return NUFFT_OK;
        } else {
            c2<T>* rr = nullptr;
            nufft_status e = fft(true, gA, gW, +1, &rr);
            if (e != NUFFT_OK) return e;
            launch_interp<T>(pl->gs, prm.ks_solve, rr, (const c2<T>*)wt_srt, out, N, bc, s);
            return NUFFT_OK;
        }
    };
    const bool fused = sizeof(T) == 4 && fft_hooks_supported<T>(tab.fft_P);
    // selection and placement as scattering stores of the FFT passes
    const bool scatter = fft_scatter_supported<T>(tab.fft_ns) && fft_scatter_supported<T>(tab.fft_P);
    // the IDFT's last pass, x K and the DFT's first pass in one kernel
    const bool conv = scatter && fft_conv_supported<T>(tab.fft_P);
    const int64_t K0 = imod(prm.K0s, ns);
    if (prm.toeplitz && (op == OP_INV5 || op == OP_INV4)) {
        // middle stage as S_m = c_m + rho^P c_{m+P}, c = L * A (linear
        // convolution with the Lagrange coefficients, by length-ns FFTs):
        // the same operator as Eqs. 37, 30, 31 without their rho^{+-k} scalings
        c2<T>* X = nullptr;
        if (op == OP_INV5) {
            launch_spread<T>(pl->gs, prm.ks_solve, in, N, (const c2<T>*)pl->wt5_ext, gA, bc, s);
            if ((st = fft(true, gA, gW, -1, &r)) != NUFFT_OK) return st;
            X = (r == gA) ? gW : gA;
            NUFFT_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(c2<T>) * ns * bc, s));
            launch_select<T>(r, ns, X, ns, P, prm.K0s, fac1, bc, s);   // A_k, k < P (type-1, Eq. 25)
        } else {
            X = gA;
            NUFFT_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(c2<T>) * ns * bc, s));
            NUFFT_CUDA_TRY(cudaMemcpy2DAsync(X, sizeof(c2<T>) * ns, in, sizeof(c2<T>) * N, sizeof(c2<T>) * N, bc,
                                             cudaMemcpyDeviceToDevice, s));
        }
        c2<T>* Y = nullptr;
        if ((st = fft(true, X, X == gA ? gW : gA, -1, &Y)) != NUFFT_OK) return st;
        launch_pointwise<T>(Y, ns, Y, ns, ns, (const c2<T>*)pl->FL, nullptr, bc, s);
        c2<T>* c = nullptr;
        if ((st = fft(true, Y, Y == gA ? gW : gA, +1, &c)) != NUFFT_OK) return st;
        if (op == OP_INV5) {
            launch_conv_fold<T>(c, ns, P, prm.rhoP, out, N, bc, s);
        } else {
            launch_conv_fold<T>(c, ns, P, prm.rhoP, vA, P, bc, s);
            launch_place<T>(vA, P, P, prm.K0s, fac1, gA, ns, bc, s);   // type-2 of S (Eq. 39)
            if ((st = fft(true, gA, gW, +1, &r)) != NUFFT_OK) return st;
            launch_interp<T>(pl->gs, prm.ks_solve, r, (const c2<T>*)pl->wt4_srt, out, N, bc, s);
        }
        NUFFT_CUDA_TRY(cudaGetLastError());
        return NUFFT_OK;
    }
    switch (op) {
        case OP_INV5: {
            launch_spread<T>(pl->gs, prm.ks_solve, in, N, (const c2<T>*)pl->wt5_ext, gA, bc, s);
            if (scatter) {
                // grid -> FFT whose last pass keeps only the N selected
                // frequencies, deconvolved and scaled by rho^k (Eq. 37); then
                // the inverse length-N FFT with Eq. 30's x K on its stores and
                // the forward one with Eq. 31's rho^-m / N, which writes the result
                FFTHooks hs;
                hs.sop = 3; hs.K0 = K0; hs.P = P; hs.out_bs = P; hs.fac_out = fac5;
                if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_ns, gA, gW, vA, bc, -1, hs, s)) != NUFFT_OK) return st;
                if (conv) {
                    FFTHooks hc;
                    hc.sop = 2; hc.fac_out = sneg;
                    if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_conv<T>, tab.fft_P, vA, vW, vA, out, bc, +1, K, hc, s)) != NUFFT_OK) return st;
                    break;
                }
                FFTHooks h1;
                h1.sop = 1; h1.mulc = K;
                if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_P, vA, vW, vA, bc, +1, h1, s)) != NUFFT_OK) return st;
                FFTHooks h2;
                h2.sop = 2; h2.fac_out = sneg;
                if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_P, vA, vW, out, bc, -1, h2, s)) != NUFFT_OK) return st;
                break;
            }
            if (fused) {
                // grid -> FFT; then Eq. 37 (selection, deconvolution, rho^k) on
                // the loads of the inverse length-N FFT, Eq. 30 (x K) on its
                // stores, and Eq. 31 (rho^-m / N) on the stores of the forward
                // FFT, which writes the result
                if ((st = fft(true, gA, gW, -1, &r)) != NUFFT_OK) return st;
                FFTHooks h1;
                h1.lop = 1; h1.src = r; h1.src_bs = ns; h1.ns = ns; h1.K0 = prm.K0s; h1.fac_in = fac5;
                h1.sop = 1; h1.mulc = K;
                if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_P, vA, vW, vA, bc, +1, h1, s)) != NUFFT_OK) return st;
                FFTHooks h2;
                h2.sop = 2; h2.fac_out = sneg;
                if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_P, vA, vW, out, bc, -1, h2, s)) != NUFFT_OK) return st;
                break;
            }
            if ((st = fft(true, gA, gW, -1, &r)) != NUFFT_OK) return st;
            launch_select<T>(r, ns, vA, P, P, prm.K0s, fac5, bc, s);
            if ((st = middle(&r)) != NUFFT_OK) return st;
            launch_pointwise<T>(r, P, out, N, P, nullptr, sneg, bc, s);
            break;
        }
        case OP_INV4: {
            if (scatter) {
                // Eq. 37's rho^k on the loads and Eq. 30's x K on the stores of
                // the inverse FFT; the forward FFT's last pass places its
                // outputs on the grid with Eq. 31 and the deconvolution folded
                // into fac4; grid FFT; type-2; x w (Eq. 40).  With ns = 2P and
                // K0 = P/2 the placed outputs fill exactly grid indices
                // g < ns/4 and g >= 3ns/4, and the grid FFT's first pass reads
                // only those (the other half is zero and is never written);
                // otherwise the other ns - N grid points are zeroed
                const bool half = ns == 2 * P && K0 == P / 2;
                if (!half) {
                    const int64_t g0 = imod(P - K0, ns), gap = ns - P;
                    const int64_t first = std::min(gap, ns - g0);
                    if (first > 0)
                        NUFFT_CUDA_TRY(
                            cudaMemset2DAsync(gA + g0, sizeof(c2<T>) * ns, 0, sizeof(c2<T>) * first, bc, s));
                    if (gap > first)
                        NUFFT_CUDA_TRY(
                            cudaMemset2DAsync(gA, sizeof(c2<T>) * ns, 0, sizeof(c2<T>) * (gap - first), bc, s));
                }
                if (conv) {
                    FFTHooks hc;
                    hc.lop = 2; hc.fac_in = rpos;
                    hc.sop = 4; hc.K0 = K0; hc.ns = ns; hc.out_bs = ns; hc.fac_out = fac4;
                    if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_conv<T>, tab.fft_P, in, vW, vA, gA, bc, +1, K, hc, s)) != NUFFT_OK) return st;
                } else {
                    FFTHooks h1;
                    h1.lop = 2; h1.fac_in = rpos;
                    h1.sop = 1; h1.mulc = K;
                    if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_P, in, vW, vA, bc, +1, h1, s)) != NUFFT_OK) return st;
                    FFTHooks h2;
                    h2.sop = 4; h2.K0 = K0; h2.ns = ns; h2.out_bs = ns; h2.fac_out = fac4;
                    if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_P, vA, vW, gA, bc, -1, h2, s)) != NUFFT_OK) return st;
                }
                if (half) {
                    FFTHooks hg;
                    hg.lop = 3;
                    if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_ns, gA, gW, gA, bc, +1, hg, s)) != NUFFT_OK) return st;
                    r = gA;
                } else if ((st = fft(true, gA, gW, +1, &r)) != NUFFT_OK) {
                    return st;
                }
                launch_interp<T>(pl->gs, prm.ks_solve, r, (const c2<T>*)pl->wt4_srt, out, N, bc, s);
                break;
            }
            if (fused) {
                // Eq. 37's rho^k on the loads and Eq. 30's x K on the stores of
                // the inverse FFT; forward FFT; Eq. 31 and the deconvolution in
                // the placement on the grid; type-2; x w (Eq. 40)
                FFTHooks h1;
                h1.lop = 2; h1.fac_in = rpos;
                h1.sop = 1; h1.mulc = K;
                if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_P, in, vW, vA, bc, +1, h1, s)) != NUFFT_OK) return st;
                FFTHooks h2;
                if ((st = traced_fft(s, sizeof(T) == 8, fft_exec_hooked<T>, tab.fft_P, vA, gW, vW, bc, -1, h2, s)) != NUFFT_OK) return st;
                launch_place<T>(vW, P, P, prm.K0s, fac4, gA, ns, bc, s);
                if ((st = fft(true, gA, gW, +1, &r)) != NUFFT_OK) return st;
                launch_interp<T>(pl->gs, prm.ks_solve, r, (const c2<T>*)pl->wt4_srt, out, N, bc, s);
                break;
            }
            launch_pointwise<T>(in, N, vA, P, P, nullptr, rpos, bc, s);
            if ((st = middle(&r)) != NUFFT_OK) return st;
            launch_place<T>(r, P, P, prm.K0s, fac4, gA, ns, bc, s);
            if ((st = grid_to_nodes(pl->wt4_srt)) != NUFFT_OK) return st;
            break;
        }
        case OP_FWD1: {
            launch_spread<T>(pl->gs, prm.ks_solve, in, N, (const c2<T>*)pl->wt1_ext, gA, bc, s);
            if ((st = fft(true, gA, gW, -1, &r)) != NUFFT_OK) return st;
            launch_select<T>(r, ns, out, N, P, prm.K0s, fac1, bc, s);
            break;
        }
        case OP_FWD2:
        case OP_FWD2D: {
            launch_place<T>(in, N, P, prm.K0s, fac1, gA, ns, bc, s, op == OP_FWD2D);
            if ((st = grid_to_nodes(pl->wt2_srt)) != NUFFT_OK) return st;
            break;
        }
    }
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

template <typename T>
nufft_status run_op(nufft_plan_s* pl, Op op, const c2<T>* in, c2<T>* out, int64_t batch, cudaStream_t s) {
    const Params& prm = pl->prm;
    const Tables& tab = *pl->tab;
    const int64_t bc = std::min<int64_t>(batch, pl->chunk);
    Sizer z;
    z.add<c2<T>>(prm.ns * bc);
    z.add<c2<T>>(fft_work_elems(tab.fft_ns) * bc);
    z.add<c2<T>>(prm.N * bc);
    z.add<c2<T>>(fft_work_elems(tab.fft_P) * bc);
    Arena sc;
    nufft_status st = sc.reserve(z.used, s);
    if (st != NUFFT_OK) return st;
    c2<T>* gA = sc.take<c2<T>>(prm.ns * bc);
    c2<T>* gW = sc.take<c2<T>>(fft_work_elems(tab.fft_ns) * bc);
    c2<T>* vA = sc.take<c2<T>>(prm.N * bc);
    c2<T>* vW = sc.take<c2<T>>(fft_work_elems(tab.fft_P) * bc);
    for (int64_t b0 = 0; b0 < batch && st == NUFFT_OK; b0 += bc) {
        const int64_t nb = std::min(bc, batch - b0);
        st = run_chunk<T>(pl, op, in + b0 * prm.N, out + b0 * prm.N, nb, gA, gW, vA, vW, s);
    }
    sc.release();
    return st;
}

// float64 forward transforms with the plan's float64 data (kernel width of
// the plan, grid of the transforms): y = G x (type-2) or y = G^H x (type-1)
nufft_status forward64(const nufft_plan_s* pl, bool type2, const double2* x, double2* y, int64_t bc, double2* g,
                       double2* gw, cudaStream_t s) {
    const Params& prm = pl->prm;
    const Tables& tab = *pl->tab;
    const int64_t N = prm.N;
    double2* r = nullptr;
    nufft_status st;
    if (type2) {
        launch_place<double>(x, N, N, prm.K0s, tab.plan_place, g, prm.ns, bc, s);
        if ((st = traced_fft(s, true, fft_exec_dd, tab.fft_ns64, g, gw, bc, +1, s, &r, 0)) != NUFFT_OK) return st;
        launch_interp<double>(pl->gs, prm.ks_plan, r, pl->modp64_srt, y, N, bc, s);
    } else {
        launch_spread<double>(pl->gs, prm.ks_plan, x, N, pl->modm64_ext, g, bc, s);
        if ((st = traced_fft(s, true, fft_exec_dd, tab.fft_ns64, g, gw, bc, -1, s, &r, 0)) != NUFFT_OK) return st;
        launch_select<double>(r, prm.ns, y, N, N, prm.K0s, tab.plan_place, bc, s);
    }
    NUFFT_CUDA_TRY(cudaGetLastError());
    return NUFFT_OK;
}

// Sec. V refinement: x1 = inv(b); r = b - F x1 with a float64 forward F;
// x2 = x1 + inv(r).  The relative error goes from eps to about eps^2 (Eq. 46).
template <typename T>
nufft_status run_refined(nufft_plan_s* pl, Op op, const c2<T>* in, c2<T>* out, int64_t batch, cudaStream_t s) {
    nufft_status st = run_op<T>(pl, op, in, out, batch, s);
    if (st != NUFFT_OK) return st;
    const Params& prm = pl->prm;
    const Tables& tab = *pl->tab;
    const int64_t N = prm.N;
    const size_t item = sizeof(double2) * (2 * N + prm.ns + fft_work_elems(tab.fft_ns64)) + 2 * sizeof(c2<T>) * N;
    const int64_t bc = std::max<int64_t>(1, std::min<int64_t>(batch, ((int64_t)512 << 20) / (int64_t)item));
    Arena ar;
    if ((st = ar.reserve(item * bc + 8 * 256, s)) != NUFFT_OK) return st;
    double2* x64 = ar.take<double2>(N * bc);
    double2* y64 = ar.take<double2>(N * bc);
    double2* g64 = ar.take<double2>(prm.ns * bc);
    double2* w64 = ar.take<double2>(fft_work_elems(tab.fft_ns64) * bc);
    c2<T>* r = ar.take<c2<T>>(N * bc);
    c2<T>* corr = ar.take<c2<T>>(N * bc);
    for (int64_t b0 = 0; b0 < batch && st == NUFFT_OK; b0 += bc) {
        const int64_t nb = std::min(bc, batch - b0);
        const c2<T>* bin = in + b0 * N;
        c2<T>* bout = out + b0 * N;
        launch_widen<T>(bout, x64, N * nb, s);
        if ((st = forward64(pl, op == OP_INV5, x64, y64, nb, g64, w64, s)) != NUFFT_OK) break;
        launch_residual<T>(bin, y64, r, N * nb, s);
        if ((st = run_op<T>(pl, op, r, corr, nb, s)) != NUFFT_OK) break;
        launch_accumulate<T>(bout, corr, N * nb, s);
    }
    ar.release();
    return st;
}

nufft_status run_public(nufft_plan_t plan, Op op, const void* in, void* out, int64_t batch, nufft_stream_t stream) {
    if (!plan) return fail(NUFFT_ERR_ARG, "null plan");
    if (batch < 0) return fail(NUFFT_ERR_ARG, "negative batch");
    if (batch == 0) return NUFFT_OK;
    if (!in || !out) return fail(NUFFT_ERR_ARG, "null data pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = solve_elem(plan->prm) * (size_t)plan->prm.N * (size_t)batch;
    const char* ib = (const char*)in;
    const char* ob = (const char*)out;
    if (ib < ob + bytes && ob < ib + bytes) return fail(NUFFT_ERR_ARG, "input and output overlap");
    const MemLoc lin = mem_loc(in), lout = mem_loc(out);
    const bool din = lin == LOC_DEVICE, dout = lout == LOC_DEVICE;
    // pinned buffers are copied on the library's copy streams, ordered against
    // `s` by events, and the call returns without waiting; pageable buffers
    // are copied on `s` and the call waits for the result
    const bool async_host = (din || lin == LOC_PINNED) && (dout || lout == LOC_PINNED);
    CopyStreams cs;
    if (async_host && (!din || !dout)) {
        nufft_status e = copy_streams(cs);
        if (e != NUFFT_OK) return e;
    }
    const void* din_p = in;
    void* dout_p = out;
    Arena stage;
    if (!din || !dout) {
        // pinned: staging memory and input copy in the copy stream's order, so
        // the copy does not wait for the work already queued on s
        nufft_status st = stage.reserve(2 * bytes, async_host ? cs.h2d : s);
        if (st != NUFFT_OK) return st;
        char* a = stage.take<char>(bytes);
        char* b = stage.take<char>(bytes);
        if (async_host) {
            if (!din) {
                cudaError_t r = cudaMemcpyAsync(a, in, bytes, cudaMemcpyHostToDevice, cs.h2d);
                if (r != cudaSuccess) { stage.release(); return cuda_fail(r, "cudaMemcpyAsync", __FILE__, __LINE__); }
            }
            nufft_status e = order_after(s, cs.h2d);
            if (e != NUFFT_OK) { stage.release(); return e; }
        } else if (!din) {
            NUFFT_CUDA_TRY(cudaMemcpyAsync(a, in, bytes, cudaMemcpyHostToDevice, s));
        }
        if (!din) din_p = a;
        if (!dout) dout_p = b;
    }
    nufft_status st;
    const bool refined = plan->prm.refine && (op == OP_INV5 || op == OP_INV4);
    if (plan->prm.prec == NUFFT_FP64)
        st = refined ? run_refined<double>(plan, op, (const double2*)din_p, (double2*)dout_p, batch, s)
                     : run_op<double>(plan, op, (const double2*)din_p, (double2*)dout_p, batch, s);
    else
        st = refined ? run_refined<float>(plan, op, (const float2*)din_p, (float2*)dout_p, batch, s)
                     : run_op<float>(plan, op, (const float2*)din_p, (float2*)dout_p, batch, s);
    if (st == NUFFT_OK && async_host) {
        if (!dout) {
            // the copy back runs behind the transforms on the copy stream and
            // overlaps whatever is queued on s next; the staging memory is
            // freed in that stream's order
            st = order_after(cs.d2h, s);
            if (st == NUFFT_OK) {
                cudaError_t r = cudaMemcpyAsync(out, dout_p, bytes, cudaMemcpyDeviceToHost, cs.d2h);
                if (r != cudaSuccess) st = cuda_fail(r, "cudaMemcpyAsync", __FILE__, __LINE__);
            }
            stage.release_on(st == NUFFT_OK ? cs.d2h : s);
            return st;
        }
        stage.release_on(s);   // s has waited for the staged input
        return st;
    }
    if (st == NUFFT_OK && !dout) {
        NUFFT_CUDA_TRY(cudaMemcpyAsync(out, dout_p, bytes, cudaMemcpyDeviceToHost, s));
        NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    } else if (st == NUFFT_OK && !din) {
        NUFFT_CUDA_TRY(cudaStreamSynchronize(s));   // the staged input must outlive its use
    }
    if (async_host) stage.release_on(s);   // s has waited for the staged copy
    else stage.release();
    return st;
}

}  // namespace

namespace {

// grad_x[q] = -(1/2pi) sum_b Re(conj(X_b[q]) Y_b[q]) where the derivative
// type-2 is applied to `deriv_of` first: inv5 (X = u, Y = s' of S) or inv4
// (X = w' of w, Y = a).
template <typename T>
nufft_status grad_nodes_impl(nufft_plan_s* pl, int kind, const c2<T>* p1, const c2<T>* p2, int64_t batch,
                             double* gx, cudaStream_t s) {
    const int64_t N = pl->prm.N;
    Arena ar;
    nufft_status st = ar.reserve(sizeof(c2<T>) * (size_t)N * (size_t)batch + 256, s);
    if (st != NUFFT_OK) return st;
    c2<T>* d = ar.take<c2<T>>((size_t)N * (size_t)batch);
    const c2<T>* src = kind == 5 ? p2 : p1;     // inv5: S; inv4: w
    st = run_op<T>(pl, OP_FWD2D, src, d, batch, s);
    if (st == NUFFT_OK) {
        const double scale = -1.0 / 6.283185307179586476925286766559;
        if (kind == 5) launch_grad_nodes<T>(p1, d, N, batch, scale, gx, s);
        else launch_grad_nodes<T>(d, p2, N, batch, scale, gx, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "launch_grad_nodes", __FILE__, __LINE__);
    }
    ar.release();
    return st;
}

nufft_status grad_nodes_public(nufft_plan_t plan, int kind, const void* p1, const void* p2, int64_t batch,
                               double* gx, nufft_stream_t stream) {
    if (!plan) return fail(NUFFT_ERR_ARG, "null plan");
    if (batch < 1) return fail(NUFFT_ERR_ARG, "batch must be >= 1");
    if (!p1 || !p2 || !gx) return fail(NUFFT_ERR_ARG, "null data pointer");
    if (!is_device_ptr(p1) || !is_device_ptr(p2) || !is_device_ptr(gx))
        return fail(NUFFT_ERR_ARG, "node gradients need device buffers");
    cudaStream_t s = (cudaStream_t)stream;
    if (plan->prm.prec == NUFFT_FP64)
        return grad_nodes_impl<double>(plan, kind, (const double2*)p1, (const double2*)p2, batch, gx, s);
    return grad_nodes_impl<float>(plan, kind, (const float2*)p1, (const float2*)p2, batch, gx, s);
}

}  // namespace

extern "C" {

nufft_status nufft_plan(int64_t N, const double* x, double tol, int prec, nufft_stream_t stream, nufft_plan_t* plan) {
    return nufft_plan_ex(N, x, tol, prec, nullptr, stream, plan);
}

static nufft_status plan_impl(int64_t N, const double* x, double tol, int prec, const nufft_params_t* params,
                              nufft_stream_t stream, nufft_plan_t* plan, const double2* Ksv, const double2* Dsv);

nufft_status nufft_plan_ex(int64_t N, const double* x, double tol, int prec, const nufft_params_t* params,
                           nufft_stream_t stream, nufft_plan_t* plan) {
    return plan_impl(N, x, tol, prec, params, stream, plan, nullptr, nullptr);
}

nufft_status nufft_plan_save(nufft_plan_t plan, void* K, void* D, nufft_stream_t stream) {
    if (!plan || !K || !D) return fail(NUFFT_ERR_ARG, "null argument");
    if (!is_device_ptr(K) || !is_device_ptr(D)) return fail(NUFFT_ERR_ARG, "nufft_plan_save needs device buffers");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b = sizeof(double2) * (size_t)plan->prm.N;
    NUFFT_CUDA_TRY(cudaMemcpyAsync(K, plan->K64, b, cudaMemcpyDeviceToDevice, s));
    NUFFT_CUDA_TRY(cudaMemcpyAsync(D, plan->D64, b, cudaMemcpyDeviceToDevice, s));
    return NUFFT_OK;
}

nufft_status nufft_plan_restore(int64_t N, const double* x, double tol, int prec, const nufft_params_t* params,
                                const void* K, const void* D, nufft_stream_t stream, nufft_plan_t* plan) {
    if (!K || !D) return fail(NUFFT_ERR_ARG, "null saved-quantity pointer");
    if (prec & NUFFT_TOEPLITZ) return fail(NUFFT_ERR_ARG, "nufft_plan_restore: NUFFT_TOEPLITZ plans cannot be restored");
    if (!is_device_ptr(K) || !is_device_ptr(D)) return fail(NUFFT_ERR_ARG, "nufft_plan_restore needs device buffers");
    return plan_impl(N, x, tol, prec, params, stream, plan, (const double2*)K, (const double2*)D);
}

static nufft_status plan_impl(int64_t N, const double* x, double tol, int prec, const nufft_params_t* params,
                              nufft_stream_t stream, nufft_plan_t* plan, const double2* Ksv, const double2* Dsv) {
    if (!plan) return fail(NUFFT_ERR_ARG, "null plan output pointer");
    *plan = nullptr;
    if (N < 1 || N > ((int64_t)1 << 28)) return fail(NUFFT_ERR_ARG, "N = %lld out of range [1, 2^28]", (long long)N);
    if (!x) return fail(NUFFT_ERR_ARG, "null node pointer");
    const bool refine = (prec & NUFFT_REFINE) != 0;
    const bool defer = (prec & NUFFT_DEFER_CHECK) != 0;
    const bool toeplitz = (prec & NUFFT_TOEPLITZ) != 0;
    prec &= ~(NUFFT_REFINE | NUFFT_DEFER_CHECK | NUFFT_TOEPLITZ);
    if (prec != NUFFT_FP32 && prec != NUFFT_FP64)
        return fail(NUFFT_ERR_ARG,
                    "precision %d is not NUFFT_FP32/NUFFT_FP64 (optionally | NUFFT_REFINE | NUFFT_DEFER_CHECK | "
                    "NUFFT_TOEPLITZ)", prec);
    if (!(tol > 0.0) || !std::isfinite(tol) || tol > 0.1) return fail(NUFFT_ERR_ARG, "tol %g out of range (0, 0.1]", tol);
    Params prm;
    nufft_status st = choose_params(N, tol, prec, prm);
    if (st != NUFFT_OK) return st;
    nufft_params_t tuned;
    if (!params) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_tuned.find(std::make_tuple(N, prec, tol));
        if (it != g_tuned.end()) { tuned = it->second; params = &tuned; }
    }
    if ((st = apply_params(params, prm)) != NUFFT_OK) return st;
    prm.refine = refine;
    prm.toeplitz = toeplitz;
    if (refine) prm.halo = std::max(prm.ks_solve.w, prm.ks_plan.w);
    int dev = 0;
    NUFFT_CUDA_TRY(cudaGetDevice(&dev));
    init_pool_once();
    nufft_status st0 = plan_kernels_init();
    if (st0 != NUFFT_OK) return st0;
    cudaStream_t s = (cudaStream_t)stream;
    nufft_plan_s* pl = new nufft_plan_s();
    pl->prm = prm;
    pl->stream = s;
    if ((st = get_tables(prm, s, pl->tab)) != NUFFT_OK) { delete pl; return st; }
    // right-hand sides per pass: keep the transforms' scratch near 256 MiB
    const int64_t item = per_item_elems(pl) * (int64_t)solve_elem(prm);
    pl->chunk = std::max<int64_t>(1, ((int64_t)256 << 20) / std::max<int64_t>(1, item));
    // nodes on the device (host arrays are staged)
    const double* xd = x;
    Arena xs;
    const MemLoc xl = mem_loc(x);
    if (xl != LOC_DEVICE) {
        // pinned nodes travel on the host-to-device copy stream (not behind
        // copies queued on s), pageable ones on s
        CopyStreams cs;
        cudaStream_t cp = s;
        if (xl == LOC_PINNED) {
            if ((st = copy_streams(cs)) != NUFFT_OK) { delete pl; return st; }
            cp = cs.h2d;
        }
        if ((st = xs.reserve(sizeof(double) * N, cp)) != NUFFT_OK) { delete pl; return st; }
        double* d = xs.take<double>(N);
        cudaError_t e = cudaMemcpyAsync(d, x, sizeof(double) * N, cudaMemcpyHostToDevice, cp);
        if (e != cudaSuccess) { xs.release(); delete pl; return cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__); }
        if (cp != s && (st = order_after(s, cp)) != NUFFT_OK) { xs.release(); delete pl; return st; }
        xd = d;
    }
    st = run_plan(pl, xd, Ksv, Dsv);
    xs.release_on(s);
    if (st == NUFFT_OK) st = plan_dup_queue(pl);
    if (st == NUFFT_OK && !defer) st = plan_dup_check(pl);
    if (st != NUFFT_OK) {
        pl->mem.release();
        cudaStreamSynchronize(s);
        plan_dup_release(pl);
        delete pl;
        return st;
    }
    *plan = pl;
    return NUFFT_OK;
}

nufft_status nufft_plan_check(nufft_plan_t plan) {
    if (!plan) return fail(NUFFT_ERR_ARG, "null plan");
    return plan_dup_check(plan);
}

nufft_status nufft_inv5(nufft_plan_t plan, const void* f, void* c, int64_t batch, nufft_stream_t stream) {
    return run_public(plan, OP_INV5, f, c, batch, stream);
}
nufft_status nufft_inv4(nufft_plan_t plan, const void* A, void* a, int64_t batch, nufft_stream_t stream) {
    return run_public(plan, OP_INV4, A, a, batch, stream);
}
nufft_status nufft_fwd1(nufft_plan_t plan, const void* a, void* A, int64_t batch, nufft_stream_t stream) {
    return run_public(plan, OP_FWD1, a, A, batch, stream);
}
nufft_status nufft_fwd2(nufft_plan_t plan, const void* c, void* f, int64_t batch, nufft_stream_t stream) {
    return run_public(plan, OP_FWD2, c, f, batch, stream);
}

nufft_status nufft_fwd2_deriv(nufft_plan_t plan, const void* c, void* f, int64_t batch, nufft_stream_t stream) {
    return run_public(plan, OP_FWD2D, c, f, batch, stream);
}

nufft_status nufft_inv5_grad_nodes(nufft_plan_t plan, const void* u, const void* S, int64_t batch, double* grad_x,
                                   nufft_stream_t stream) {
    return grad_nodes_public(plan, 5, u, S, batch, grad_x, stream);
}

nufft_status nufft_inv4_grad_nodes(nufft_plan_t plan, const void* w, const void* a, int64_t batch, double* grad_x,
                                   nufft_stream_t stream) {
    return grad_nodes_public(plan, 4, w, a, batch, grad_x, stream);
}

// ------------------------------------------------------- parameter tuner ---
namespace {

// deterministic CN(0,1)-like test vectors (a linear congruential generator;
// their statistics do not matter, only that the round trip exercises every
// coefficient)
void test_vector(std::vector<double>& v, uint64_t seed) {
    uint64_t z = seed * 0x9E3779B97F4A7C15ull + 1;
    for (auto& e : v) {
        z = z * 6364136223846793005ull + 1442695040888963407ull;
        e = ((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5) * 2.449489742783178;   // unit variance
    }
}

double rel_err(const std::vector<double>& a, const std::vector<double>& b) {
    double num = 0, den = 0;
    for (size_t i = 0; i < a.size(); ++i) { num += (a[i] - b[i]) * (a[i] - b[i]); den += b[i] * b[i]; }
    return std::sqrt(num / den);
}

}  // namespace

nufft_status nufft_plan_tune(int64_t N, const double* x, double tol, int prec, int64_t batch, nufft_stream_t stream,
                             nufft_params_t* best, double* best_ms) {
    if (!best) return fail(NUFFT_ERR_ARG, "null result pointer");
    if (prec != NUFFT_FP32 && prec != NUFFT_FP64) return fail(NUFFT_ERR_ARG, "precision %d", prec);
    if (batch < 1 || batch > 1024) return fail(NUFFT_ERR_ARG, "batch %lld out of range [1, 1024]", (long long)batch);
    if (!(tol > 0.0) || !std::isfinite(tol) || tol > 0.1) return fail(NUFFT_ERR_ARG, "tol %g out of range (0, 0.1]", tol);
    cudaStream_t s = (cudaStream_t)stream;
    Params dflt;
    nufft_status st = choose_params(N, tol, prec, dflt);
    if (st != NUFFT_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_tuned.erase(std::make_tuple(N, prec, tol));
    }
    // candidates: truncation 0.4 gamma^-eta (Sec. V, measured law) at most tol / 10
    std::vector<nufft_params_t> cands;
    const double gammas32[] = {30, 100, 300, 1000, 3000};
    const double gammas64[] = {100, 1000, 10000};
    const int wps32[] = {10, 12};
    // (the smallest such eta per gamma: a larger eta only costs plan time)
    auto min_eta = [&](double g) {
        int eta = 1;
        while (eta < 24 && 0.4 * std::pow(g, -eta) > tol / 10) ++eta;
        return eta;
    };
    if (prec == NUFFT_FP32) {
        for (double g : gammas32)
            for (int wp : wps32) cands.push_back({g, min_eta(g), wp, 0});
    } else {
        for (double g : gammas64) cands.push_back({g, min_eta(g), 0, 0});
    }
    const size_t es = prec == NUFFT_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t n = (size_t)N * (size_t)batch;
    std::vector<double> c(2 * n), back(2 * n);
    test_vector(c, 1);
    std::vector<char> hc(es * n), hb(es * n);
    auto to_data = [&](const std::vector<double>& v, std::vector<char>& h) {
        if (prec == NUFFT_FP64) std::memcpy(h.data(), v.data(), es * n);
        else for (size_t i = 0; i < 2 * n; ++i) reinterpret_cast<float*>(h.data())[i] = (float)v[i];
    };
    auto from_data = [&](const std::vector<char>& h, std::vector<double>& v) {
        if (prec == NUFFT_FP64) std::memcpy(v.data(), h.data(), es * n);
        else for (size_t i = 0; i < 2 * n; ++i) v[i] = reinterpret_cast<const float*>(h.data())[i];
    };
    to_data(c, hc);
    if (prec == NUFFT_FP32) from_data(hc, c);   // compare against the rounded input
    Arena buf;
    if ((st = buf.reserve(3 * es * n + 512, s)) != NUFFT_OK) return st;
    char* d0 = buf.take<char>(es * n);
    char* d1 = buf.take<char>(es * n);
    char* d2 = buf.take<char>(es * n);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bool found = false;
    double best_t = 1e300;
    for (const nufft_params_t& q : cands) {
        nufft_plan_t pl = nullptr;
        st = nufft_plan_ex(N, x, tol, prec, &q, stream, &pl);
        if (st == NUFFT_ERR_DUP_NODES) break;
        if (st != NUFFT_OK) continue;
        // a posteriori accuracy: c -> type-2 -> inv5 and c -> type-1 -> inv4
        double err = 0;
        cudaError_t ce = cudaMemcpyAsync(d0, hc.data(), es * n, cudaMemcpyHostToDevice, s);
        for (int kind = 5; kind >= 4 && ce == cudaSuccess && st == NUFFT_OK; --kind) {
            st = kind == 5 ? nufft_fwd2(pl, d0, d1, batch, stream) : nufft_fwd1(pl, d0, d1, batch, stream);
            if (st == NUFFT_OK) st = kind == 5 ? nufft_inv5(pl, d1, d2, batch, stream) : nufft_inv4(pl, d1, d2, batch, stream);
            if (st == NUFFT_OK) ce = cudaMemcpyAsync(hb.data(), d2, es * n, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce == cudaSuccess && st == NUFFT_OK) {
                from_data(hb, back);
                err = std::max(err, rel_err(back, c));
            }
        }
        if (ce != cudaSuccess) { nufft_destroy(pl); buf.release(); cudaEventDestroy(e0); cudaEventDestroy(e1);
                                 return cuda_fail(ce, "tuner", __FILE__, __LINE__); }
        nufft_destroy(pl);
        if (st != NUFFT_OK || !(err <= tol / 2)) { st = NUFFT_OK; continue; }
        // time: plan + inv5 + inv4 on `batch` vectors, best of 3
        double t = 1e300;
        for (int r = 0; r < 3 && st == NUFFT_OK; ++r) {
            cudaEventRecord(e0, s);
            st = nufft_plan_ex(N, x, tol, prec | NUFFT_DEFER_CHECK, &q, stream, &pl);
            if (st == NUFFT_OK) st = nufft_inv5(pl, d1, d2, batch, stream);
            if (st == NUFFT_OK) st = nufft_inv4(pl, d1, d2, batch, stream);
            cudaEventRecord(e1, s);
            if (pl) nufft_destroy(pl);
            pl = nullptr;
            if (cudaEventSynchronize(e1) != cudaSuccess) st = NUFFT_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, (double)ms);
        }
        if (st != NUFFT_OK) { st = NUFFT_OK; continue; }
        if (t < best_t) { best_t = t; *best = q; found = true; }
    }
    buf.release();
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != NUFFT_OK) return st;
    if (!found) return fail(NUFFT_ERR_ACCURACY, "no candidate parameter set met tol %g on these nodes", tol);
    if (best->w_plan <= 0) best->w_plan = dflt.ks_plan.w;
    if (best->w_solve <= 0) best->w_solve = dflt.ks_solve.w;
    if (best_ms) *best_ms = best_t;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_tuned[std::make_tuple(N, prec, tol)] = *best;
    return NUFFT_OK;
}

nufft_status nufft_destroy(nufft_plan_t plan) {
    if (!plan) return NUFFT_OK;
    // stream-ordered release: work already queued on the plan's stream keeps
    // its buffers; kernels hold no reference to the host-side object
    plan->mem.release();
    plan_dup_release(plan);
    delete plan;
    return NUFFT_OK;
}

nufft_status nufft_plan_set_batch_chunk(nufft_plan_t plan, int64_t chunk) {
    if (!plan || chunk < 1) return fail(NUFFT_ERR_ARG, "bad plan or chunk");
    plan->chunk = chunk;
    return NUFFT_OK;
}

nufft_status nufft_plan_info(nufft_plan_t plan, nufft_plan_info_t* info) {
    if (!plan || !info) return fail(NUFFT_ERR_ARG, "null argument");
    const Params& p = plan->prm;
    info->N = p.N; info->prec = p.prec; info->tol = p.tol;
    info->gamma = p.gamma; info->a = p.a; info->rho = p.rho;
    info->eta = p.eta; info->R = p.R;
    info->grid_solve = p.ns; info->grid_plan = p.ns;
    info->w_solve = p.ks_solve.w; info->w_plan = p.ks_plan.w;
    info->beta_solve = p.ks_solve.beta; info->beta_plan = p.ks_plan.beta;
    info->batch_chunk = plan->chunk;
    return NUFFT_OK;
}

nufft_status nufft_plan_export(nufft_plan_t plan, int which, void* dst, nufft_stream_t stream) {
    if (!plan || !dst) return fail(NUFFT_ERR_ARG, "null argument");
    const double2* src = which == 0 ? plan->K64 : which == 1 ? plan->D64 : which == 2 ? plan->w64 : nullptr;
    if (!src) return fail(NUFFT_ERR_ARG, "unknown export %d", which);
    cudaStream_t s = (cudaStream_t)stream;
    NUFFT_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double2) * plan->prm.N, cudaMemcpyDefault, s));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(s));
    return NUFFT_OK;
}

nufft_status nufft_stream_check(nufft_stream_t stream) {
    CopyStreams cs;
    nufft_status st = copy_streams(cs);
    if (st != NUFFT_OK) return st;
    NUFFT_CUDA_TRY(cudaStreamSynchronize(cs.h2d));
    NUFFT_CUDA_TRY(cudaStreamSynchronize(cs.d2h));
    return fft_wait_status((cudaStream_t)stream);
}

nufft_status nufft_cache_clear(void) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache.clear();
    g_tuned.clear();
    return NUFFT_OK;
}

const char* nufft_status_string(nufft_status st) {
    switch (st) {
        case NUFFT_OK: return "NUFFT_OK";
        case NUFFT_ERR_ARG: return "NUFFT_ERR_ARG";
        case NUFFT_ERR_DUP_NODES: return "NUFFT_ERR_DUP_NODES";
        case NUFFT_ERR_ALLOC: return "NUFFT_ERR_ALLOC";
        case NUFFT_ERR_CUDA: return "NUFFT_ERR_CUDA";
        case NUFFT_ERR_TIMEOUT: return "NUFFT_ERR_TIMEOUT";
        case NUFFT_ERR_ACCURACY: return "NUFFT_ERR_ACCURACY";
    }
    return "unknown status";
}

const char* nufft_last_error_message(void) { return g_msg; }

// Test hook (not part of the public header): run the library's FFT of length
// n on `batch` contiguous device vectors in place (prec 1: complex64, 2:
// complex128, 3: complex128 data through the double-float FFT; dir -1
// forward, +1 inverse, unnormalised).  Synchronises.
nufft_status nufft_debug_fft(int64_t n, int prec, int dir, int64_t batch, void* buf, nufft_stream_t stream) {
    if (n < 1 || batch < 1 || !buf || prec < 1 || prec > 3 || (dir != 1 && dir != -1))
        return fail(NUFFT_ERR_ARG, "bad FFT test arguments");
    cudaStream_t s = (cudaStream_t)stream;
    FFTPlan p;
    nufft_status st = fft_make(p, n, prec, s);
    if (st != NUFFT_OK) return st;
    const size_t es = prec >= 2 ? sizeof(double2) : sizeof(float2);
    void* work = nullptr;
    NUFFT_CUDA_TRY(cudaMalloc(&work, es * (size_t)fft_work_elems(p) * (size_t)batch));
    void* res = nullptr;
    if (prec == 3) st = fft_exec_dd(p, (double2*)buf, (double2*)work, batch, dir, s, (double2**)&res);
    else if (prec == 2) st = fft_exec<double>(p, (double2*)buf, (double2*)work, batch, dir, s, (double2**)&res);
    else st = fft_exec<float>(p, (float2*)buf, (float2*)work, batch, dir, s, (float2**)&res);
    if (st == NUFFT_OK && res != buf)
        st = cudaMemcpyAsync(buf, res, es * n * batch, cudaMemcpyDeviceToDevice, s) == cudaSuccess ? NUFFT_OK : NUFFT_ERR_CUDA;
    cudaStreamSynchronize(s);
    cudaFree(work);
    return st;
}

// Test hook (not part of the public header): make the next `count` device
// allocations fail with NUFFT_ERR_ALLOC, to exercise the error paths without
// exhausting the device.
void nufft_debug_fail_allocs(int count) { g_fail_allocs = count; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free type-5 inverse.
//
// nufft_inv5 takes its scratch (the oversampled grid and the FFT work
// vectors) from the stream-ordered pool on every call.  Some callers cannot
// allocate device memory when they transform: real-time loops and embedded
// runtimes that forbid allocation after set-up, code that runs under a
// device-memory budget enforced by an external allocator, or hosts that only
// hand out pre-registered buffers.  nufft_inv5_noalloc runs the same kernels
// one right-hand side at a time on a fixed scratch array that is part of the
// library image (a file-scope __device__ array, resident on every GPU that
// loads the library until the process exits).  The plan itself is still made
// by nufft_plan, at set-up time.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 8 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in for the symbol and must never be
// handed to a kernel.  Resolved once per device, with that device current.
nufft_status noalloc_scratch(void** out) {
    int dev = 0;
    NUFFT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NUFFT_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return NUFFT_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Offsets into the static scratch for one right-hand side.  The inverse uses
// the grid, its FFT work vector and the two length-N vectors (region U).  A
// refined plan (Sec. V, Eqs. 44-46) also needs the float64 copy of the first
// solution, the float64 forward transform of it, the residual and the
// correction; the float64 forward's grid and work vector are only live
// between the two inverses, so they share region U with the inverse's
// buffers, and the correction reuses the float64 copy's slot once the
// forward transform has read it.
struct NoAllocLayout {
    size_t gA = 0, gW = 0, vA = 0, vW = 0;      // inverse (region U)
    size_t g64 = 0, gw64 = 0;                   // float64 forward (region U)
    size_t x64 = 0, y64 = 0, r = 0;             // refinement
    size_t corr = 0;                            // = x64
    size_t need = 0;
};

NoAllocLayout noalloc_layout(const nufft_plan_s* pl) {
    const Params& prm = pl->prm;
    const Tables& tab = *pl->tab;
    const size_t es = solve_elem(prm);
    NoAllocLayout L;
    size_t u = 0;
    L.gA = u; u += round256(es * prm.ns);
    L.gW = u; u += round256(es * fft_work_elems(tab.fft_ns));
    L.vA = u; u += round256(es * prm.N);
    L.vW = u; u += round256(es * fft_work_elems(tab.fft_P));
    if (!prm.refine) {
        L.need = u;
        return L;
    }
    size_t f = 0;
    L.g64 = f; f += round256(sizeof(double2) * prm.ns);
    L.gw64 = f; f += round256(sizeof(double2) * fft_work_elems(tab.fft_ns64));
    size_t q = std::max(u, f);
    L.x64 = q; q += round256(sizeof(double2) * prm.N);
    L.y64 = q; q += round256(sizeof(double2) * prm.N);
    L.r = q; q += round256(es * prm.N);
    L.corr = L.x64;
    L.need = q;
    return L;
}

template <typename T>
nufft_status inv5_noalloc_impl(nufft_plan_s* pl, const c2<T>* in, c2<T>* out, int64_t batch, char* scratch,
                               cudaStream_t s) {
    const Params& prm = pl->prm;
    const int64_t N = prm.N;
    const NoAllocLayout L = noalloc_layout(pl);
    c2<T>* gA = reinterpret_cast<c2<T>*>(scratch + L.gA);
    c2<T>* gW = reinterpret_cast<c2<T>*>(scratch + L.gW);
    c2<T>* vA = reinterpret_cast<c2<T>*>(scratch + L.vA);
    c2<T>* vW = reinterpret_cast<c2<T>*>(scratch + L.vW);
    for (int64_t b = 0; b < batch; ++b) {
        const c2<T>* bin = in + b * N;
        c2<T>* bout = out + b * N;
        nufft_status st = run_chunk<T>(pl, OP_INV5, bin, bout, 1, gA, gW, vA, vW, s);
        if (st != NUFFT_OK) return st;
        if (!prm.refine) continue;
        // Sec. V refinement as in nufft_inv5: x2 = x1 + inv(b - G x1), the
        // residual from a float64 type-2 transform with the plan's float64 data
        double2* x64 = reinterpret_cast<double2*>(scratch + L.x64);
        double2* y64 = reinterpret_cast<double2*>(scratch + L.y64);
        c2<T>* r = reinterpret_cast<c2<T>*>(scratch + L.r);
        c2<T>* corr = reinterpret_cast<c2<T>*>(scratch + L.corr);
        launch_widen<T>(bout, x64, N, s);
        st = forward64(pl, true, x64, y64, 1, reinterpret_cast<double2*>(scratch + L.g64),
                       reinterpret_cast<double2*>(scratch + L.gw64), s);
        if (st != NUFFT_OK) return st;
        launch_residual<T>(bin, y64, r, N, s);
        if ((st = run_chunk<T>(pl, OP_INV5, r, corr, 1, gA, gW, vA, vW, s)) != NUFFT_OK) return st;
        launch_accumulate<T>(bout, corr, N, s);
        NUFFT_CUDA_TRY(cudaGetLastError());
    }
    return NUFFT_OK;
}

}  // namespace

extern "C" nufft_status nufft_inv5_noalloc(nufft_plan_t plan, const void* f, void* c, int64_t batch,
                                           nufft_stream_t stream) {
    if (!plan) return fail(NUFFT_ERR_ARG, "null plan");
    if (batch < 0) return fail(NUFFT_ERR_ARG, "negative batch");
    if (batch == 0) return NUFFT_OK;
    if (!f || !c) return fail(NUFFT_ERR_ARG, "null data pointer");
    const Params& prm = plan->prm;
    const size_t es = solve_elem(prm);
    const size_t need = noalloc_layout(plan).need;
    if (need > kNoAllocScratchBytes)
        return fail(NUFFT_ERR_ARG,
                    "nufft_inv5_noalloc: N = %lld%s needs %zu bytes of scratch per right-hand side, more than the "
                    "%zu-byte static scratch; use nufft_inv5", (long long)prm.N, prm.refine ? " (refined)" : "",
                    need, kNoAllocScratchBytes);
    const size_t bytes = es * (size_t)prm.N * (size_t)batch;
    const char* ib = (const char*)f;
    const char* ob = (const char*)c;
    if (ib < ob + bytes && ob < ib + bytes) return fail(NUFFT_ERR_ARG, "input and output overlap");
    if (!is_device_ptr(f) || !is_device_ptr(c))
        return fail(NUFFT_ERR_ARG, "nufft_inv5_noalloc needs device buffers (host buffers would need staging memory)");
    void* scratch = nullptr;
    nufft_status st = noalloc_scratch(&scratch);
    if (st != NUFFT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (prm.prec == NUFFT_FP64)
        return inv5_noalloc_impl<double>(plan, (const double2*)f, (double2*)c, batch, (char*)scratch, s);
    return inv5_noalloc_impl<float>(plan, (const float2*)f, (float2*)c, batch, (char*)scratch, s);
}

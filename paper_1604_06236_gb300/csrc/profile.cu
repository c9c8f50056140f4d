// Kernel-level tracing: every launch of the library is counted; when
// enabled, each launch is bracketed by CUDA events on its own stream and
// attributed to a kernel class with its algorithmic byte count.  The passes of
// one FFT, which run back to back, share one pair of events (LaunchGroup).
#include "internal.h"

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

namespace nufft45 {

namespace {
struct Rec { int kind; cudaEvent_t a, b; double bytes; long long n; };
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free;
std::atomic<long long> g_launches{0};
thread_local LaunchGroup* t_group = nullptr;

cudaEvent_t get_event() {
    if (!g_free.empty()) { cudaEvent_t e = g_free.back(); g_free.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

const char* kind_name(int k) {
    static const char* names[] = {"fft_pass", "spread", "interp", "select", "place", "pointwise",
                                  "geometry", "plan_table", "plan_stage", "bluestein",
                                  "fft_pass_f64", "spread_f64", "interp_f64", "select_f64", "place_f64",
                                  "pointwise_f64", "geometry_f64", "plan_table_f64", "plan_stage_f64",
                                  "bluestein_f64"};
    return (k >= 0 && k < 2 * K_COUNT) ? names[k] : "unknown";
}

Launch::Launch(cudaStream_t s, int kind, double bytes, bool f64) : s_(s), kind_(kind + (f64 ? K_COUNT : 0)), bytes_(bytes) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_on) {
        if (t_group && t_group->join(s_, kind_, bytes_)) return;
        std::lock_guard<std::mutex> lk(g_mu);
        a_ = get_event();
        b_ = get_event();
        cudaEventRecord(a_, s_);
    }
}

Launch::~Launch() {
    if (a_) {
        cudaEventRecord(b_, s_);
        std::lock_guard<std::mutex> lk(g_mu);
        g_recs.push_back(Rec{kind_, a_, b_, bytes_, 1});
    }
}

LaunchGroup::LaunchGroup(cudaStream_t s, int kind, bool f64) : s_(s), kind_(kind + (f64 ? K_COUNT : 0)) {
    outer_ = (t_group == nullptr);
    if (outer_) t_group = this;
}

LaunchGroup::~LaunchGroup() {
    if (!outer_) return;
    close();
    t_group = nullptr;
}

bool LaunchGroup::join(cudaStream_t s, int kind, double bytes) {
    if (s != s_ || kind != kind_) {
        close();   // the run ends before a launch of another kind
        return false;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!a_) {
        a_ = get_event();
        cudaEventRecord(a_, s_);
        n_ = 0;
        bytes_ = 0;
    }
    n_ += 1;
    bytes_ += bytes;
    return true;
}

void LaunchGroup::close() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = get_event();
    cudaEventRecord(b, s_);
    g_recs.push_back(Rec{kind_, a_, b, bytes_, n_});
    a_ = nullptr;
}

// independent FMA chains: kChains accumulators per thread, so the pipe,
// not the dependency latency, sets the rate; the result is stored so the
// chains stay live
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T b, T c, T* __restrict__ out) {
    T acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], b, c);
        }
    }
    T sum = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) sum += acc[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

template <typename T>
nufft_status measure_fma(double* tflops, cudaStream_t s) {
    int dev = 0, sms = 0;
    NUFFT_CUDA_TRY(cudaGetDevice(&dev));
    NUFFT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 8 * sms, threads = 256;
    // enough work for a launch of a few milliseconds at either rate
    const int iters = sizeof(T) == 4 ? 4096 : 64;
    T* out = nullptr;
    NUFFT_CUDA_TRY(cudaMallocAsync(&out, sizeof(T) * blocks * threads, s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b just below 1 and c tiny keep the chains finite
    k_fma_rate<T><<<blocks, threads, 0, s>>>(iters, (T)0.999999, (T)1e-7, out);
    cudaEventRecord(e0, s);
    k_fma_rate<T><<<blocks, threads, 0, s>>>(iters, (T)0.999999, (T)1e-7, out);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, s);
    if (e != cudaSuccess) return cuda_fail(e, "fma rate", __FILE__, __LINE__);
    g_launches.fetch_add(2, std::memory_order_relaxed);
    const double fmas = (double)blocks * threads * iters * 8.0 * kChains;
    *tflops = ms > 0.f ? 2.0 * fmas / ((double)ms * 1e-3) / 1e12 : 0.0;
    return NUFFT_OK;
}

}  // namespace nufft45

using namespace nufft45;

extern "C" {

nufft_status nufft_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (on) {
        for (auto& r : g_recs) { g_free.push_back(r.a); g_free.push_back(r.b); }
        g_recs.clear();
    }
    g_on = on != 0;
    return NUFFT_OK;
}

int64_t nufft_launch_count(void) { return (int64_t)g_launches.load(); }

nufft_status nufft_measure_fma(int prec, double* tflops, nufft_stream_t stream) {
    if (!tflops) return fail(NUFFT_ERR_ARG, "null result pointer");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == NUFFT_FP32) return measure_fma<float>(tflops, s);
    if (prec == NUFFT_FP64) return measure_fma<double>(tflops, s);
    return fail(NUFFT_ERR_ARG, "precision %d is neither NUFFT_FP32 nor NUFFT_FP64", prec);
}

nufft_status nufft_profile_read(nufft_profile_entry_t* out, int cap, int* count) {
    if (!out || !count || cap < 0) return fail(NUFFT_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(g_mu);
    nufft_profile_entry_t acc[2 * K_COUNT];
    std::memset(acc, 0, sizeof(acc));
    for (int k = 0; k < 2 * K_COUNT; ++k) std::strncpy(acc[k].name, kind_name(k), sizeof(acc[k].name) - 1);
    for (auto& r : g_recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize", __FILE__, __LINE__);
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime", __FILE__, __LINE__);
        acc[r.kind].launches += r.n;
        acc[r.kind].ms += ms;
        acc[r.kind].bytes += r.bytes;
    }
    int n = 0;
    for (int k = 0; k < 2 * K_COUNT && n < cap; ++k)
        if (acc[k].launches > 0) out[n++] = acc[k];
    *count = n;
    return NUFFT_OK;
}

}  // extern "C"

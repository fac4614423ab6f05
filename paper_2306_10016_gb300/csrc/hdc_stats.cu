// hdc_stats.cu -- launch counters and per-kernel CUDA-event timing.
//
// The bench reads, for each kernel of the path, how many launches ran, their
// summed device time (from events recorded on the launch stream around each
// launch) and the model flops / algorithmic bytes they processed.  Timing is
// off by default; counting is always on.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <mutex>
#include <unordered_set>
#include <vector>

#include "hdc.h"
#include "hdc_internal.h"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace hdc {

namespace {
struct KStat {
    int64_t launches = 0;
    double flops = 0.0, bytes = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};
std::mutex g_mu;
KStat g_k[K_COUNT];
std::atomic<int> g_timing{ 0 };
std::atomic<int64_t> g_total{ 0 };
std::vector<cudaEvent_t> g_pool;
// Events recorded inside a stream capture: an instantiated graph keeps
// recording them on every replay for as long as it lives, and the library
// cannot tell when the caller destroys it.  They are therefore never handed
// out again (a recycled one would be recorded by the graph and by a later
// launch alike, and both timings would be wrong); they stay allocated until
// the process exits.
std::unordered_set<cudaEvent_t> g_captured;
const char* g_names[K_COUNT] = { "k_twiddle", "k_residue_rows", "k_fold_fft_cols", "k_ifft_cols", "k_unfold",
                                 "k_batched", "k_ifft_unfold_cols", "k_fold_fft_cols_tma", "k_conv_cluster",
                                 "k_hermitian_rows" };

// Inside a stream capture an event record must be an external record node
// for the event to carry a time stamp when the graph replays.
void record(cudaEvent_t e, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive) {
        g_captured.insert(e);
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    } else
        cudaEventRecord(e, st);
}

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
} // namespace

double fft_flops(double n) { return n > 1 ? 5.0 * n * std::log2(n) : 0.0; }

LaunchScope::LaunchScope(int k, cudaStream_t s, double flops, double bytes) : kid(k), st(s), e0(nullptr)
{
    g_total.fetch_add(1);
    std::lock_guard<std::mutex> lk(g_mu);
    g_k[kid].launches += 1;
    g_k[kid].flops += flops;
    g_k[kid].bytes += bytes;
    if (g_timing.load()) {
        e0 = take_event();
        if (e0) record(e0, st);
    }
}

LaunchScope::~LaunchScope()
{
    if (!e0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e1 = take_event();
    if (!e1) return;
    record(e1, st);
    g_k[kid].ev.emplace_back(e0, e1);
}

} // namespace hdc

using namespace hdc;

HDC_EXPORT int hdc_stats_reset(void)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& k : g_k) {
        for (auto& pr : k.ev)
            for (cudaEvent_t e : { pr.first, pr.second })
                if (!g_captured.count(e)) g_pool.push_back(e);
        k = KStat();
    }
    g_total.store(0);
    return HDC_OK;
}

HDC_EXPORT int hdc_stats_timing(int on)
{
    g_timing.store(on ? 1 : 0);
    return HDC_OK;
}

HDC_EXPORT int hdc_stats_kernel_count(void) { return K_COUNT; }

HDC_EXPORT const char* hdc_stats_kernel_name(int id) { return (id >= 0 && id < K_COUNT) ? g_names[id] : "?"; }

HDC_EXPORT int64_t hdc_stats_total_launches(void) { return g_total.load(); }

HDC_EXPORT int hdc_stats_get(int id, int64_t* launches, double* ms, double* flops, double* bytes)
{
    if (id < 0 || id >= K_COUNT) return HDC_ERR_PARAM;
    std::lock_guard<std::mutex> lk(g_mu);
    const KStat& k = g_k[id];
    double tot = 0.0;
    for (auto& pr : k.ev) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pr.first, pr.second) != cudaSuccess) return HDC_ERR_CUDA;
        tot += t;
    }
    if (launches) *launches = k.launches;
    if (ms) *ms = tot;
    if (flops) *flops = k.flops;
    if (bytes) *bytes = k.bytes;
    return HDC_OK;
}

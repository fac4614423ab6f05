// hdc_tune.cu -- parameter search and plans.
//
// The exhaustive tuner is the grid search of Section 4.2 (A0): enumerate the
// valid (m, p, q, D) of an axis, time each candidate on the device, keep the
// fastest.  For N dimensions it uses the separability argument of the same
// section: each axis is searched with the other axes held at their current
// best, one axis after the other, so the cost is the sum and not the product
// of the per-axis candidate counts.  The timing score is the whole
// convolution (Section 4.3 times only the forward routine; a GPU launch
// sequence has no separable forward cost worth scoring on its own).
//
// Candidates of an axis: for each q, the m of the form 2^a 3^b 5^c 7^d that
// pad M least (the three smallest >= ceil(M/q), the next power of two and the
// next 3 * 2^k), with p = ceil(L/m), q = ceil(M/m), D = q; kept when their
// model flops F1 = q (15 m log2 m + 6 m + 24 L) + 2 L are within max_ratio of
// the smallest F1 of the axis (m >= m_min).  The fastest few m are then
// re-timed with D in {1, 2, 4, ...} below q.
//
// Plans remember the chosen parameters; a text tuning database keyed by
// (device, dtype, batch, dims, L, M) caches search results across runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hdc.h"
#include "hdc_internal.h"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

double model_flops_axis(int64_t L, int64_t m, int64_t q)
{
    const double md = (double)m;
    const double lg = m > 1 ? std::log2(md) : 0.0;
    return (double)q * (15.0 * md * lg + 6.0 * md + 24.0 * (double)L) + 2.0 * (double)L;
}

int64_t next_pow2_times(int64_t n, int64_t base)
{
    int64_t v = base;
    while (v < n) v *= 2;
    return v;
}

// For every q, the m that pad M least: the three smallest good sizes
// >= ceil(M/q), the next power of two and the next 3 * 2^k (sizes whose FFTs
// use the largest radices).  q grows until even the fold/unfold term
// 24 q L alone exceeds max_ratio times the best model flops seen.
std::vector<hdc_tuple> candidates(int64_t L, int64_t M, int dtype, double max_ratio, int64_t m_min)
{
    std::vector<hdc_tuple> out;
    if (m_min < 1) m_min = 1;
    // an axis too short for any m >= m_min keeps its explicit size
    const int64_t top = hdc_next_good_size(M);
    if (top > 0 && top < m_min) m_min = top;
    double best = 1e300;
    std::vector<int64_t> ms;
    for (int64_t q = 1;; ++q) {
        const int64_t lo = (M + q - 1) / q;
        if (lo < m_min && q > 1) break;
        if (24.0 * (double)q * (double)L > max_ratio * best) break;
        int64_t m = lo;
        for (int k = 0; k < 3; ++k) {
            m = hdc_next_good_size(m);
            if (m < 1) break;
            ms.push_back(m);
            best = std::min(best, model_flops_axis(L, m, (M + m - 1) / m));
            ++m;
        }
        ms.push_back(next_pow2_times(lo, 1));
        ms.push_back(next_pow2_times(lo, 3));
    }
    std::sort(ms.begin(), ms.end());
    ms.erase(std::unique(ms.begin(), ms.end()), ms.end());
    for (int64_t m : ms) {
        if (m < m_min) continue;
        int64_t p = 0, q = 0, D = 0;
        if (hdc_validate_axis(L, M, m, 0, 0, 0, dtype, &p, &q, &D) != HDC_OK) continue;
        hdc_tuple t;
        t.m = m; t.p = p; t.q = q; t.D = q;
        t.model_flops = model_flops_axis(L, m, q);
        t.ms = -1.0;
        out.push_back(t);
    }
    if (out.empty()) return out;
    best = out[0].model_flops;
    for (auto& t : out) best = std::min(best, t.model_flops);
    // explicit padding (m = nextgood(M), q = 1) is always a candidate: it is
    // the path the hybrid choice has to beat, and the search keeps it on ties
    std::vector<hdc_tuple> kept;
    for (auto& t : out)
        if (t.model_flops <= max_ratio * best || (t.q == 1 && t.m == top)) kept.push_back(t);
    std::sort(kept.begin(), kept.end(),
              [](const hdc_tuple& a, const hdc_tuple& b) { return a.model_flops < b.model_flops; });
    return kept;
}

// Candidates of axis i of a dims-axis problem: an axis with inner axes runs
// its transform in one column tile, so m above hdc_max_outer_fft_size is
// dropped there (it would be rejected with HDC_ERR_UNSUPPORTED_SIZE).
int64_t transform_size(const hdc_tuple& t) { return t.m; }
int64_t transform_size(const hdc_unequal_tuple& t) { return t.m * t.lam; }

template <class Tup> std::vector<Tup> drop_outer_oversize(std::vector<Tup> c, int i, int dims, int dtype)
{
    if (i >= dims - 1) return c;
    const int64_t lim = hdc_max_outer_fft_size(dtype);
    std::vector<Tup> out;
    for (const auto& t : c)
        if (transform_size(t) <= lim) out.push_back(t);
    return out;
}

std::vector<hdc_tuple> axis_candidates(const int64_t* L, const int64_t* M, int i, int dims, int dtype,
                                       double max_ratio, int64_t m_min)
{
    return drop_outer_oversize(candidates(L[i], M[i], dtype, max_ratio, m_min), i, dims, dtype);
}

std::string device_key()
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
    std::string s = pr.name;
    for (auto& c : s)
        if (c == ' ') c = '_';
    return s;
}

std::mutex g_db_mu;

std::string db_key(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch)
{
    std::string k = "v1 " + device_key() + " " + std::to_string(dtype) + " " + std::to_string(batch) + " " +
                    std::to_string(dims);
    for (int i = 0; i < dims; ++i) k += " " + std::to_string(L[i]);
    for (int i = 0; i < dims; ++i) k += " " + std::to_string(M[i]);
    return k;
}

bool db_lookup(const char* path, const std::string& key, int dims, hdc_tuple* best)
{
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lk(g_db_mu);
    FILE* fp = fopen(path, "r");
    if (!fp) return false;
    char line[4096];
    bool found = false;
    while (fgets(line, sizeof line, fp)) {
        char* bar = strchr(line, '|');
        if (!bar) continue;
        std::string k(line, bar - line);
        while (!k.empty() && k.back() == ' ') k.pop_back();
        if (k != key) continue;
        // record: per axis "m p q D", then the time
        const char* s = bar + 1;
        hdc_tuple t[HDC_MAX_DIMS];
        bool ok = true;
        int used = 0;
        for (int i = 0; i < dims && ok; ++i) {
            long long m, p, q, D;
            if (sscanf(s, " %lld %lld %lld %lld%n", &m, &p, &q, &D, &used) != 4) ok = false;
            s += used;
            t[i].m = m; t[i].p = p; t[i].q = q; t[i].D = D;
            t[i].model_flops = 0.0;
        }
        double ms = -1.0;
        if (ok && sscanf(s, " %lf", &ms) != 1) ok = false;
        if (!ok) continue; // a corrupt line is skipped, never trusted
        for (int i = 0; i < dims; ++i) {
            t[i].ms = ms;
            best[i] = t[i];
        }
        found = true; // the last matching record wins
    }
    fclose(fp);
    return found;
}

void db_store(const char* path, const std::string& key, int dims, const hdc_tuple* best)
{
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lk(g_db_mu);
    FILE* fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s |", key.c_str());
    for (int i = 0; i < dims; ++i)
        fprintf(fp, " %lld %lld %lld %lld", (long long)best[i].m, (long long)best[i].p, (long long)best[i].q,
                (long long)best[i].D);
    fprintf(fp, " %.6f\n", best[0].ms);
    fclose(fp);
}


// ----------------------------------------------------- unequal lengths

double model_flops_uneq(int64_t Lf, int64_t Lg, int64_t mg, int64_t lam, int64_t qg)
{
    const double md = (double)mg, mf = (double)(mg / lam);
    const double lg = mg > 1 ? std::log2(md) : 0.0, lf = mf > 1 ? std::log2(mf) : 0.0;
    return (double)qg * (10.0 * md * lg + 5.0 * lam * mf * lf + 6.0 * md +
                         8.0 * ((double)Lg + (double)lam * Lf + (double)Lg)) +
           2.0 * (double)Lg;
}

std::vector<hdc_unequal_tuple> candidates_uneq(int64_t Lf, int64_t Lg, int64_t M, int dtype, double max_ratio,
                                               int64_t m_min)
{
    std::vector<hdc_unequal_tuple> out;
    if (m_min < 1) m_min = 1;
    const int64_t top = hdc_next_good_size(M);
    if (top > 0 && top < m_min) m_min = top;
    double best = 1e300;
    std::vector<int64_t> ms;
    for (int64_t q = 1;; ++q) {
        const int64_t lo = (M + q - 1) / q;
        if (lo < m_min && q > 1) break;
        if (16.0 * (double)q * (double)Lg > max_ratio * best) break;
        int64_t m = lo;
        for (int k = 0; k < 3; ++k) {
            m = hdc_next_good_size(m);
            if (m < 1) break;
            ms.push_back(m);
            best = std::min(best, model_flops_uneq(Lf, Lg, m, 1, (M + m - 1) / m));
            ++m;
        }
        ms.push_back(next_pow2_times(lo, 1));
        ms.push_back(next_pow2_times(lo, 3));
    }
    std::sort(ms.begin(), ms.end());
    ms.erase(std::unique(ms.begin(), ms.end()), ms.end());
    for (int64_t mg : ms) {
        if (mg < m_min) continue;
        for (int64_t base : { (int64_t)1, (int64_t)3 })
            for (int64_t lam = base; lam <= mg; lam *= 2) {
                if (mg % lam) continue;
                // f's cost 5 mg log2(m) + 8 lam Lf per residue of g is least
                // near m = mg / lam ~ Lf: keep lam = 1 and m in [Lf/2, 2 Lf]
                const int64_t mf = mg / lam;
                if (lam > 1 && (2 * mf < Lf || mf > 2 * Lf)) continue;
                int64_t pf = 0, pg = 0, qg = 0, D = 0;
                if (hdc_validate_unequal_axis(Lf, Lg, M, mg / lam, lam, 0, dtype, &pf, &pg, &qg, &D) != HDC_OK)
                    continue;
                hdc_unequal_tuple t;
                t.m = mg / lam; t.lam = lam; t.q = qg; t.D = qg;
                t.model_flops = model_flops_uneq(Lf, Lg, mg, lam, qg);
                t.ms = -1.0;
                out.push_back(t);
            }
    }
    if (out.empty()) return out;
    best = out[0].model_flops;
    for (auto& t : out) best = std::min(best, t.model_flops);
    std::vector<hdc_unequal_tuple> kept;
    for (auto& t : out)
        if (t.model_flops <= max_ratio * best) kept.push_back(t);
    std::sort(kept.begin(), kept.end(), [](const hdc_unequal_tuple& a, const hdc_unequal_tuple& b) {
        return a.model_flops < b.model_flops;
    });
    return kept;
}

std::string db_key_uneq(int dims, const int64_t* Lf, const int64_t* Lg, const int64_t* M, int dtype, int64_t batch)
{
    std::string k = "u1 " + device_key() + " " + std::to_string(dtype) + " " + std::to_string(batch) + " " +
                    std::to_string(dims);
    for (int i = 0; i < dims; ++i) k += " " + std::to_string(Lf[i]);
    for (int i = 0; i < dims; ++i) k += " " + std::to_string(Lg[i]);
    for (int i = 0; i < dims; ++i) k += " " + std::to_string(M[i]);
    return k;
}

// Records "key | m lam q D (per axis) ms"; the last valid matching line wins.
bool db_lookup_uneq(const char* path, const std::string& key, int dims, hdc_unequal_tuple* best)
{
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lk(g_db_mu);
    FILE* fp = fopen(path, "r");
    if (!fp) return false;
    char line[4096];
    bool found = false;
    while (fgets(line, sizeof line, fp)) {
        char* bar = strchr(line, '|');
        if (!bar) continue;
        std::string k(line, bar - line);
        while (!k.empty() && k.back() == ' ') k.pop_back();
        if (k != key) continue;
        const char* s = bar + 1;
        hdc_unequal_tuple t[HDC_MAX_DIMS];
        bool ok = true;
        int used = 0;
        for (int i = 0; i < dims && ok; ++i) {
            long long m, lam, q, D;
            if (sscanf(s, " %lld %lld %lld %lld%n", &m, &lam, &q, &D, &used) != 4) ok = false;
            s += used;
            t[i].m = m; t[i].lam = lam; t[i].q = q; t[i].D = D;
            t[i].model_flops = 0.0;
        }
        double ms = -1.0;
        if (ok && sscanf(s, " %lf", &ms) != 1) ok = false;
        if (!ok) continue;
        for (int i = 0; i < dims; ++i) {
            t[i].ms = ms;
            best[i] = t[i];
        }
        found = true;
    }
    fclose(fp);
    return found;
}

void db_store_uneq(const char* path, const std::string& key, int dims, const hdc_unequal_tuple* best)
{
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lk(g_db_mu);
    FILE* fp = fopen(path, "a");
    if (!fp) return;
    fprintf(fp, "%s |", key.c_str());
    for (int i = 0; i < dims; ++i)
        fprintf(fp, " %lld %lld %lld %lld", (long long)best[i].m, (long long)best[i].lam, (long long)best[i].q,
                (long long)best[i].D);
    fprintf(fp, " %.6f\n", best[0].ms);
    fclose(fp);
}


int resolve_M_uneq(int dims, const int64_t* Lf, const int64_t* Lg, const int64_t* M, int64_t* Mo)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !Lf || !Lg) return HDC_ERR_PARAM;
    for (int i = 0; i < dims; ++i) {
        if (Lf[i] < 1 || Lg[i] < 1) return HDC_ERR_PARAM;
        Mo[i] = (M && M[i] > 0) ? M[i] : Lf[i] + Lg[i] - 1;
        if (Mo[i] < Lf[i] + Lg[i] - 1) return HDC_ERR_ALIAS;
    }
    return HDC_OK;
}

// Median device time (ms) of one call, timed the way the throughput
// measurement times a step: `warmup` eager calls on `st` (they also make the
// candidate's twiddle tables), then the call captured once in a CUDA graph
// on a private stream and replayed `reps` times, each replay preceded by a
// write of a 256 MiB buffer that evicts the 129 MB L2 (outside the events).
// Eager timing would add the host's launch gaps to small problems and keep
// their data in L2, which favoured tuples the replayed step then ran slower.
// call(s) enqueues the convolution on stream s.  < 0 if a call fails.
constexpr double kMinSampleMs = 1.0;
constexpr int kMaxReps = 41;

template <class CallFn> double median_ms(CallFn call, int warmup, int reps, cudaStream_t st)
{
    // a search may allocate: the candidates' twiddle tables are made as the
    // first call of each one meets them
    hdc::TableScope tables(hdc::kTablesCreate);
    for (int w = 0; w < warmup; ++w)
        if (call(st) != HDC_OK) return -1.0;
    size_t fbytes = 0;
    void* flush = hdc::tuning_flush_buffer(&fbytes);
    if (!flush || cudaStreamSynchronize(st) != cudaSuccess) return -1.0;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return -1.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double res = -1.0;
    std::vector<float> ts;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const int rc = call(cs);
        const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
        if (rc != HDC_OK || ec != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) goto done;
    } else {
        goto done;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    if (cudaGraphLaunch(exec, cs) != cudaSuccess) goto done;   // the first replay uploads the graph
    // `reps` replays, then more (up to kMaxReps) until about kMinSampleMs of
    // replays are in the sample: a 30 us call timed 5 times is a 0.15 ms
    // sample, whose median moves by a few percent from run to run
    {
        int want = reps;
        for (int r = 0; r < want; ++r) {
            if (cudaMemsetAsync(flush, r & 0xff, fbytes, cs) != cudaSuccess) break;
            cudaEventRecord(e0, cs);
            if (cudaGraphLaunch(exec, cs) != cudaSuccess) break;
            cudaEventRecord(e1, cs);
            if (cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ts.push_back(ms);
            if (r + 1 == reps && reps > 0) {
                std::vector<float> tmp(ts);
                std::sort(tmp.begin(), tmp.end());
                const double med = tmp[tmp.size() / 2];
                if (med > 0.0 && med * reps < kMinSampleMs)
                    want = (int)std::min<double>(kMaxReps, std::ceil(kMinSampleMs / med));
            }
        }
        if ((int)ts.size() == want && want > 0) {
            std::sort(ts.begin(), ts.end());
            res = ts[ts.size() / 2];
        }
    }
done:
    cudaStreamSynchronize(cs);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    return res;
}

// Median device time of one configuration of each kind (ms), or < 0 on error.
double time_config(int dims, const void* f, const void* g, void* h, const int64_t* L, const int64_t* M,
                   const hdc_tuple* t, int dtype, int64_t batch, void* ws, size_t ws_bytes, int warmup, int reps,
                   cudaStream_t st)
{
    int64_t m[HDC_MAX_DIMS], p[HDC_MAX_DIMS], q[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) { m[i] = t[i].m; p[i] = t[i].p; q[i] = t[i].q; D[i] = t[i].D; }
    size_t need = 0;
    if (hdc_workspace_size(dims, L, M, m, p, q, D, dtype, batch, 0, &need) != HDC_OK || need > ws_bytes) return -1.0;
    return median_ms(
        [&](cudaStream_t s) { return hdc_convnd(dims, f, g, h, L, M, m, p, q, D, 0, dtype, batch, ws, ws_bytes, s); },
        warmup, reps, st);
}

double time_config_uneq(int dims, const void* f, const void* g, void* h, const int64_t* Lf, const int64_t* Lg,
                        const int64_t* M, const hdc_unequal_tuple* t, int dtype, int64_t batch, void* ws,
                        size_t ws_bytes, int warmup, int reps, cudaStream_t st)
{
    int64_t m[HDC_MAX_DIMS], lam[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) { m[i] = t[i].m; lam[i] = t[i].lam; D[i] = t[i].D; }
    size_t need = 0;
    if (hdc_workspace_size_unequal(dims, Lf, Lg, M, m, lam, D, nullptr, nullptr, dtype, batch, &need) != HDC_OK ||
        need > ws_bytes)
        return -1.0;
    return median_ms(
        [&](cudaStream_t s) {
            return hdc_convnd_unequal(dims, f, g, h, Lf, Lg, M, m, lam, D, nullptr, nullptr, dtype, batch, ws,
                                      ws_bytes, s);
        },
        warmup, reps, st);
}

double time_config_multi(int dims, int n, int op, const void* const* xs, void* h, const int64_t* L,
                         const int64_t* M, const hdc_tuple* t, int dtype, int64_t batch, void* ws, size_t ws_bytes,
                         int warmup, int reps, cudaStream_t st)
{
    int64_t m[HDC_MAX_DIMS], p[HDC_MAX_DIMS], q[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) { m[i] = t[i].m; p[i] = t[i].p; q[i] = t[i].q; D[i] = t[i].D; }
    size_t need = 0;
    if (hdc_workspace_size_multi(dims, n, op, L, M, m, p, q, D, dtype, batch, &need) != HDC_OK || need > ws_bytes)
        return -1.0;
    return median_ms(
        [&](cudaStream_t s) {
            return hdc_convnd_multi(dims, n, op, xs, h, L, M, m, p, q, D, dtype, batch, ws, ws_bytes, s);
        },
        warmup, reps, st);
}

double time_config_real(int dims, const void* f, const void* g, void* h, const int64_t* L, const int64_t* M,
                        const hdc_tuple* t, int dtype, int64_t batch, void* ws, size_t ws_bytes, int warmup, int reps,
                        cudaStream_t st)
{
    int64_t m[HDC_MAX_DIMS], p[HDC_MAX_DIMS], q[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) { m[i] = t[i].m; p[i] = t[i].p; q[i] = t[i].q; D[i] = t[i].D; }
    size_t need = 0;
    if (hdc_workspace_size_real(dims, L, M, m, p, q, D, dtype, batch, &need) != HDC_OK || need > ws_bytes)
        return -1.0;
    return median_ms(
        [&](cudaStream_t s) { return hdc_convnd_real(dims, f, g, h, L, M, m, p, q, D, dtype, batch, ws, ws_bytes, s); },
        warmup, reps, st);
}

// The separable search of Section 4.2 over per-axis candidate lists c[ax]
// (tuples with q, D and ms fields): axes from the last to the first, each
// swept with the others at their best so far (the smallest model flops to
// start), then the three fastest of the axis re-timed with D = 1, 2, 4, ...
// below q.  time(t) is the median ms of the whole call for the tuple array
// t (< 0: unusable).  trials (cap records of dims tuples) gets every timed
// configuration, *ntrials their count.
// Explicit padding (Section 3.1): one residue of the whole padded length.
bool is_explicit(const hdc_tuple& t) { return t.q == 1; }
bool is_explicit(const hdc_unequal_tuple& t) { return t.q == 1 && t.lam == 1; }
// A faster tuple replaces explicit padding only if it is faster by more than
// this fraction (the spread of the median of replays is below it).
constexpr double kTieFraction = 0.01;

template <class Tup, class TimeFn>
int separable_search(int dims, const std::vector<Tup>* c, TimeFn time, Tup* best, Tup* trials, int64_t cap,
                     int64_t* ntrials)
{
    Tup cur[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) cur[i] = c[i][0];
    int64_t nt = 0;
    auto record = [&](const Tup* t, double ms) {
        if (trials && nt < cap) {
            for (int i = 0; i < dims; ++i) {
                trials[nt * dims + i] = t[i];
                trials[nt * dims + i].ms = ms;
            }
        }
        ++nt;
    };
    double best_ms = -1.0;
    for (int ax = dims - 1; ax >= 0; --ax) {
        std::vector<std::pair<double, Tup>> timed;
        for (const auto& cand : c[ax]) {
            Tup t[HDC_MAX_DIMS];
            for (int i = 0; i < dims; ++i) t[i] = cur[i];
            t[ax] = cand;
            const double ms = time(t);
            if (ms < 0) continue;
            record(t, ms);
            timed.emplace_back(ms, cand);
        }
        if (timed.empty()) return HDC_ERR_CUDA;
        std::sort(timed.begin(), timed.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        // the leaders and the explicit candidate are timed twice more,
        // interleaved, and keep the median of their three times: a drift of
        // the clock or of the memory system during the search then cannot
        // decide between them
        {
            std::vector<size_t> again;
            for (size_t k = 0; k < timed.size(); ++k)
                if (k < 4 || is_explicit(timed[k].second)) again.push_back(k);
            std::vector<std::vector<double>> smp(again.size());
            for (size_t j = 0; j < again.size(); ++j) smp[j].push_back(timed[again[j]].first);
            for (int round = 0; round < 2; ++round)
                for (size_t j = 0; j < again.size(); ++j) {
                    Tup t[HDC_MAX_DIMS];
                    for (int i = 0; i < dims; ++i) t[i] = cur[i];
                    t[ax] = timed[again[j]].second;
                    const double ms = time(t);
                    if (ms < 0) continue;
                    record(t, ms);
                    smp[j].push_back(ms);
                }
            for (size_t j = 0; j < again.size(); ++j) {
                std::sort(smp[j].begin(), smp[j].end());
                timed[again[j]].first = smp[j][(smp[j].size() - 1) / 2];
            }
            std::sort(timed.begin(), timed.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        }
        Tup bax = timed[0].second;
        double bms = timed[0].first;
        for (size_t k = 0; k < timed.size() && k < 3; ++k) {
            const Tup base = timed[k].second;
            for (int64_t Dv = 1; Dv < base.q; Dv *= 2) {
                Tup t[HDC_MAX_DIMS];
                for (int i = 0; i < dims; ++i) t[i] = cur[i];
                t[ax] = base;
                t[ax].D = Dv;
                const double ms = time(t);
                if (ms < 0) continue;
                record(t, ms);
                if (ms < bms) { bms = ms; bax = t[ax]; }
            }
        }
        // ties go to explicit padding
        for (const auto& tm : timed)
            if (is_explicit(tm.second) && tm.first <= bms * (1.0 + kTieFraction)) {
                bax = tm.second;
                bms = tm.first;
                break;
            }
        cur[ax] = bax;
        best_ms = bms;
    }
    for (int i = 0; i < dims; ++i) {
        best[i] = cur[i];
        best[i].ms = best_ms;
    }
    if (ntrials) *ntrials = nt;
    return HDC_OK;
}

} // namespace

// ------------------------------------------------------------------ ABI

HDC_EXPORT int hdc_tune_candidates(int64_t L, int64_t M, int dtype, double max_ratio, int64_t m_min,
                                   hdc_tuple* out, int64_t cap, int64_t* n)
{
    if (!n || L < 1 || M < 2 * L - 1 || max_ratio < 1.0) return L >= 1 && M < 2 * L - 1 ? HDC_ERR_ALIAS : HDC_ERR_PARAM;
    if (dtype != HDC_C64 && dtype != HDC_C128) return HDC_ERR_DTYPE;
    auto c = candidates(L, M, dtype, max_ratio, m_min);
    *n = (int64_t)c.size();
    for (int64_t i = 0; i < cap && i < (int64_t)c.size(); ++i) out[i] = c[i];
    return HDC_OK;
}

HDC_EXPORT int hdc_tune_workspace_size(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch,
                                       double max_ratio, int64_t m_min, size_t* bytes)
{
    if (!bytes || dims < 1 || dims > HDC_MAX_DIMS || !L || !M) return HDC_ERR_PARAM;
    // per-axis worst case: the largest workspace any single-axis candidate
    // (with every D) needs while the other axes take their worst candidate
    std::vector<hdc_tuple> c[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) {
        c[i] = axis_candidates(L, M, i, dims, dtype, max_ratio, m_min);
        if (c[i].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
    }
    size_t worst = 0;
    int64_t m[HDC_MAX_DIMS], p[HDC_MAX_DIMS], q[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    // enumerate the product (small: a few dozen per axis)
    int64_t idx[HDC_MAX_DIMS] = { 0, 0, 0 };
    while (true) {
        for (int i = 0; i < dims; ++i) {
            const hdc_tuple& t = c[i][idx[i]];
            m[i] = t.m; p[i] = t.p; q[i] = t.q; D[i] = t.q;
        }
        size_t b = 0;
        if (hdc_workspace_size(dims, L, M, m, p, q, D, dtype, batch, 0, &b) == HDC_OK) worst = std::max(worst, b);
        int k = dims - 1;
        while (k >= 0 && ++idx[k] == (int64_t)c[k].size()) idx[k--] = 0;
        if (k < 0) break;
    }
    *bytes = worst;
    return HDC_OK;
}

HDC_EXPORT int hdc_tune_convnd(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch,
                               const void* f, const void* g, void* h, void* ws, size_t ws_bytes, int warmup,
                               int reps, double max_ratio, int64_t m_min, void* stream, hdc_tuple* best,
                               hdc_tuple* trials, int64_t cap, int64_t* ntrials)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !L || !M || !best || !f || !g || !h || reps < 1) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<hdc_tuple> c[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) {
        if (M[i] < 2 * L[i] - 1) return HDC_ERR_ALIAS;
        c[i] = axis_candidates(L, M, i, dims, dtype, max_ratio, m_min);
        if (c[i].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
    }
    return separable_search<hdc_tuple>(
        dims, c,
        [&](const hdc_tuple* t) {
            return time_config(dims, f, g, h, L, M, t, dtype, batch, ws, ws_bytes, warmup, reps, st);
        },
        best, trials, cap, ntrials);
}

HDC_EXPORT int hdc_tune_conv1d(int64_t L, int64_t M, int dtype, int64_t batch, const void* f, const void* g,
                               void* h, void* ws, size_t ws_bytes, int warmup, int reps, double max_ratio,
                               int64_t m_min, void* stream, hdc_tuple* best, hdc_tuple* trials, int64_t cap,
                               int64_t* ntrials)
{
    return hdc_tune_convnd(1, &L, &M, dtype, batch, f, g, h, ws, ws_bytes, warmup, reps, max_ratio, m_min, stream,
                           best, trials, cap, ntrials);
}

HDC_EXPORT int hdc_tune_unequal_candidates(int64_t Lf, int64_t Lg, int64_t M, int dtype, double max_ratio,
                                           int64_t m_min, hdc_unequal_tuple* out, int64_t cap, int64_t* n)
{
    if (!n || max_ratio < 1.0) return HDC_ERR_PARAM;
    if (dtype != HDC_C64 && dtype != HDC_C128) return HDC_ERR_DTYPE;
    int64_t Mv = 0;
    int rc = resolve_M_uneq(1, &Lf, &Lg, &M, &Mv);
    if (rc != HDC_OK) return rc;
    auto c = candidates_uneq(Lf, Lg, Mv, dtype, max_ratio, m_min);
    *n = (int64_t)c.size();
    for (int64_t i = 0; i < cap && i < (int64_t)c.size(); ++i) out[i] = c[i];
    return HDC_OK;
}

HDC_EXPORT int hdc_tune_unequal_workspace_size(int dims, const int64_t* Lf, const int64_t* Lg, const int64_t* M,
                                               int dtype, int64_t batch, double max_ratio, int64_t m_min,
                                               size_t* bytes)
{
    if (!bytes) return HDC_ERR_PARAM;
    int64_t Mv[HDC_MAX_DIMS];
    int rc = resolve_M_uneq(dims, Lf, Lg, M, Mv);
    if (rc != HDC_OK) return rc;
    std::vector<hdc_unequal_tuple> c[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) {
        c[i] = drop_outer_oversize(candidates_uneq(Lf[i], Lg[i], Mv[i], dtype, max_ratio, m_min), i, dims, dtype);
        if (c[i].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
    }
    size_t worst = 0;
    int64_t m[HDC_MAX_DIMS], lam[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    int64_t idx[HDC_MAX_DIMS] = { 0, 0, 0 };
    while (true) {
        for (int i = 0; i < dims; ++i) {
            const hdc_unequal_tuple& t = c[i][idx[i]];
            m[i] = t.m; lam[i] = t.lam; D[i] = t.q;
        }
        size_t b = 0;
        if (hdc_workspace_size_unequal(dims, Lf, Lg, Mv, m, lam, D, nullptr, nullptr, dtype, batch, &b) == HDC_OK)
            worst = std::max(worst, b);
        int k = dims - 1;
        while (k >= 0 && ++idx[k] == (int64_t)c[k].size()) idx[k--] = 0;
        if (k < 0) break;
    }
    *bytes = worst;
    return HDC_OK;
}

HDC_EXPORT int hdc_tune_unequal(int dims, const int64_t* Lf, const int64_t* Lg, const int64_t* M, int dtype,
                                int64_t batch, const void* f, const void* g, void* h, void* ws, size_t ws_bytes,
                                int warmup, int reps, double max_ratio, int64_t m_min, const char* tuning_db,
                                void* stream, hdc_unequal_tuple* best, hdc_unequal_tuple* trials, int64_t cap,
                                int64_t* ntrials)
{
    if (!best || !f || !g || !h || reps < 1) return HDC_ERR_PARAM;
    int64_t Mv[HDC_MAX_DIMS];
    int rc = resolve_M_uneq(dims, Lf, Lg, M, Mv);
    if (rc != HDC_OK) return rc;
    const std::string key = db_key_uneq(dims, Lf, Lg, Mv, dtype, batch);
    if (db_lookup_uneq(tuning_db, key, dims, best)) {
        if (ntrials) *ntrials = 0;
        return HDC_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<hdc_unequal_tuple> c[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) {
        c[i] = drop_outer_oversize(candidates_uneq(Lf[i], Lg[i], Mv[i], dtype, max_ratio, m_min), i, dims, dtype);
        if (c[i].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
    }
    rc = separable_search<hdc_unequal_tuple>(
        dims, c,
        [&](const hdc_unequal_tuple* t) {
            return time_config_uneq(dims, f, g, h, Lf, Lg, Mv, t, dtype, batch, ws, ws_bytes, warmup, reps, st);
        },
        best, trials, cap, ntrials);
    if (rc != HDC_OK) return rc;
    db_store_uneq(tuning_db, key, dims, best);
    return HDC_OK;
}

HDC_EXPORT int hdc_tune_multi_workspace_size(int dims, int n, int op, const int64_t* L, const int64_t* M,
                                             int dtype, int64_t batch, double max_ratio, int64_t m_min,
                                             size_t* bytes)
{
    if (!bytes || dims < 1 || dims > HDC_MAX_DIMS || !L || !M) return HDC_ERR_PARAM;
    std::vector<hdc_tuple> c[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) {
        c[i] = axis_candidates(L, M, i, dims, dtype, max_ratio, m_min);
        if (c[i].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
    }
    size_t worst = 0;
    int64_t m[HDC_MAX_DIMS], p[HDC_MAX_DIMS], q[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    int64_t idx[HDC_MAX_DIMS] = { 0, 0, 0 };
    while (true) {
        for (int i = 0; i < dims; ++i) {
            const hdc_tuple& t = c[i][idx[i]];
            m[i] = t.m; p[i] = t.p; q[i] = t.q; D[i] = t.q;
        }
        size_t b = 0;
        if (hdc_workspace_size_multi(dims, n, op, L, M, m, p, q, D, dtype, batch, &b) == HDC_OK)
            worst = std::max(worst, b);
        int k = dims - 1;
        while (k >= 0 && ++idx[k] == (int64_t)c[k].size()) idx[k--] = 0;
        if (k < 0) break;
    }
    *bytes = worst;
    return HDC_OK;
}

HDC_EXPORT int hdc_tune_multi(int dims, int n, int op, const int64_t* L, const int64_t* M, int dtype,
                              int64_t batch, const void* const* inputs, void* h, void* ws, size_t ws_bytes,
                              int warmup, int reps, double max_ratio, int64_t m_min, void* stream, hdc_tuple* best,
                              hdc_tuple* trials, int64_t cap, int64_t* ntrials)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !L || !M || !best || !inputs || !h || reps < 1) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<hdc_tuple> c[HDC_MAX_DIMS];
    const int fold = op == HDC_MULTI_PRODUCT ? n : 2;
    for (int i = 0; i < dims; ++i) {
        if (M[i] < fold * (L[i] - 1) + 1) return HDC_ERR_ALIAS;
        c[i] = axis_candidates(L, M, i, dims, dtype, max_ratio, m_min);
        if (c[i].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
    }
    return separable_search<hdc_tuple>(
        dims, c,
        [&](const hdc_tuple* t) {
            return time_config_multi(dims, n, op, inputs, h, L, M, t, dtype, batch, ws, ws_bytes, warmup, reps, st);
        },
        best, trials, cap, ntrials);
}

HDC_EXPORT int hdc_tune_real_workspace_size(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch,
                                            double max_ratio, int64_t m_min, size_t* bytes)
{
    if (!bytes || dims < 1 || dims > HDC_MAX_DIMS || !L || !M) return HDC_ERR_PARAM;
    std::vector<hdc_tuple> c[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) {
        c[i] = candidates(L[i], M[i], dtype, max_ratio, m_min);
        if (c[i].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
    }
    size_t worst = 0;
    int64_t m[HDC_MAX_DIMS], p[HDC_MAX_DIMS], q[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    int64_t idx[HDC_MAX_DIMS] = { 0, 0, 0 };
    while (true) {
        for (int i = 0; i < dims; ++i) {
            const hdc_tuple& t = c[i][idx[i]];
            m[i] = t.m; p[i] = t.p; q[i] = t.q; D[i] = t.q;
        }
        size_t b = 0;
        if (hdc_workspace_size_real(dims, L, M, m, p, q, D, dtype, batch, &b) == HDC_OK) worst = std::max(worst, b);
        int k = dims - 1;
        while (k >= 0 && ++idx[k] == (int64_t)c[k].size()) idx[k--] = 0;
        if (k < 0) break;
    }
    *bytes = worst;
    return HDC_OK;
}

HDC_EXPORT int hdc_tune_real(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch, const void* f,
                             const void* g, void* h, void* ws, size_t ws_bytes, int warmup, int reps, double max_ratio,
                             int64_t m_min, void* stream, hdc_tuple* best, hdc_tuple* trials, int64_t cap,
                             int64_t* ntrials)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !L || !M || !best || !f || !g || !h || reps < 1) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<hdc_tuple> c[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) {
        if (M[i] < 2 * L[i] - 1) return HDC_ERR_ALIAS;
        c[i] = axis_candidates(L, M, i, dims, dtype, max_ratio, m_min);
        if (c[i].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
    }
    return separable_search<hdc_tuple>(
        dims, c,
        [&](const hdc_tuple* t) {
            return time_config_real(dims, f, g, h, L, M, t, dtype, batch, ws, ws_bytes, warmup, reps, st);
        },
        best, trials, cap, ntrials);
}

// --------------------------------------------------- cheap tuners (A1)

namespace {

// SplitMix64 (Steele, Lea and Flood 2014): the seeded stream the random
// search draws its samples from.
uint64_t splitmix64_next(uint64_t* state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// n distinct entries of c drawn uniformly (partial Fisher-Yates), kept in
// model-flops order; all of c when n >= |c|.
std::vector<hdc_tuple> sample_candidates(const std::vector<hdc_tuple>& c, int64_t n, uint64_t* state)
{
    if (n >= (int64_t)c.size()) return c;
    std::vector<size_t> idx(c.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    for (int64_t k = 0; k < n; ++k) {
        const size_t j = (size_t)k + (size_t)(splitmix64_next(state) % (uint64_t)(idx.size() - (size_t)k));
        std::swap(idx[(size_t)k], idx[j]);
    }
    std::vector<size_t> pick(idx.begin(), idx.begin() + n);
    std::sort(pick.begin(), pick.end());
    std::vector<hdc_tuple> out;
    for (size_t i : pick) out.push_back(c[i]);
    return out;
}

} // namespace

HDC_EXPORT int hdc_tune_convnd_random(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch,
                                      const void* f, const void* g, void* h, void* ws, size_t ws_bytes, int warmup,
                                      int reps, double max_ratio, int64_t m_min, int64_t n_samples, uint64_t seed,
                                      void* stream, hdc_tuple* best, hdc_tuple* trials, int64_t cap,
                                      int64_t* ntrials)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !L || !M || !best || !f || !g || !h || reps < 1) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<hdc_tuple> c[HDC_MAX_DIMS];
    uint64_t state = seed;
    for (int i = 0; i < dims; ++i) {
        if (M[i] < 2 * L[i] - 1) return HDC_ERR_ALIAS;
        const auto all = axis_candidates(L, M, i, dims, dtype, max_ratio, m_min);
        if (all.empty()) return HDC_ERR_UNSUPPORTED_SIZE;
        const int64_t n = n_samples > 0 ? n_samples : std::max<int64_t>(3, ((int64_t)all.size() + 3) / 4);
        c[i] = sample_candidates(all, n, &state);
    }
    return separable_search<hdc_tuple>(
        dims, c,
        [&](const hdc_tuple* t) {
            return time_config(dims, f, g, h, L, M, t, dtype, batch, ws, ws_bytes, warmup, reps, st);
        },
        best, trials, cap, ntrials);
}

HDC_EXPORT int hdc_tune_convnd_proxy(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch,
                                     const void* f, const void* g, void* h, void* ws, size_t ws_bytes, int warmup,
                                     int reps, double max_ratio, int64_t m_min, int64_t Lproxy, void* stream,
                                     hdc_tuple* best, int64_t* ntrials)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !L || !M || !best || !f || !g || !h || reps < 1 || Lproxy < 1)
        return HDC_ERR_PARAM;
    int64_t total = 0;
    for (int ax = 0; ax < dims; ++ax) {
        if (M[ax] < 2 * L[ax] - 1) return HDC_ERR_ALIAS;
        // the rectangle: this axis at full length, every other axis cut to
        // Lproxy (with its least alias-free padding)
        int64_t Lp[HDC_MAX_DIMS], Mp[HDC_MAX_DIMS];
        for (int j = 0; j < dims; ++j) {
            const bool cut = j != ax && L[j] > Lproxy;
            Lp[j] = cut ? Lproxy : L[j];
            Mp[j] = cut ? 2 * Lproxy - 1 : M[j];
        }
        size_t need = 0;
        int rc = hdc_tune_workspace_size(dims, Lp, Mp, dtype, batch, max_ratio, m_min, &need);
        if (rc != HDC_OK) return rc;
        if (need > ws_bytes) return HDC_ERR_WORKSPACE;
        hdc_tuple pb[HDC_MAX_DIMS];
        int64_t nt = 0;
        // the rectangle's arrays are prefixes of the caller's buffers
        rc = hdc_tune_convnd(dims, Lp, Mp, dtype, batch, f, g, h, ws, ws_bytes, warmup, reps, max_ratio, m_min,
                             stream, pb, nullptr, 0, &nt);
        if (rc != HDC_OK) return rc;
        best[ax] = pb[ax];
        total += nt;
    }
    if (ntrials) *ntrials = total;
    return HDC_OK;
}

// ---------------------------------------------------------------- plans

// Search bounds of plans made with HDC_TUNE_EXHAUSTIVE: candidates within
// 1.5x of the smallest model flops, m >= 16.
constexpr double kPlanRatio = 1.5;
// timed replays per candidate (median)
constexpr int kPlanReps = 5;
constexpr int64_t kPlanMmin = 16;
// HDC_TUNE_RANDOM: a quarter of each axis' candidates (at least 3), drawn
// with this seed; HDC_TUNE_PROXY: the other axes cut to 32 points.
constexpr uint64_t kPlanSeed = 230610016ULL;
constexpr int64_t kPlanProxy = 32;

struct hdc_plan {
    int dims;
    int dtype;
    int64_t batch;
    int64_t L[HDC_MAX_DIMS], M[HDC_MAX_DIMS];
    hdc_tuple t[HDC_MAX_DIMS];
    size_t ws;
    int64_t timed; // configurations timed while the plan was made
};

// Logits of the learned predictor for every axis: features, one forward
// pass of the network on the device.
static int mlp_logits(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch, const char* path,
                      cudaStream_t st, std::vector<float>& logits)
{
    if (!path || !*path) return HDC_ERR_NOT_TUNED;
    const int nq = hdc_mlp_num_q_classes();
    hdc_mlp* net = nullptr;
    int rc = hdc_mlp_create(&net, HDC_MLP_FEATURES, HDC_MLP_HIDDEN, nq + 2);
    if (rc != HDC_OK) return rc;
    if (hdc_mlp_load(net, path) != HDC_OK) { hdc_mlp_destroy(net); return HDC_ERR_NOT_TUNED; }
    float feat[HDC_MAX_DIMS * HDC_MLP_FEATURES];
    rc = hdc_mlp_axis_features(dims, L, M, dtype, batch, feat);
    logits.assign((size_t)dims * (nq + 2), 0.f);
    float* dbuf = nullptr;
    if (rc == HDC_OK && cudaMalloc(&dbuf, sizeof(float) * (size_t)dims * (HDC_MLP_FEATURES + nq + 2)) != cudaSuccess)
        rc = HDC_ERR_ALLOC;
    if (rc == HDC_OK) {
        float* dx = dbuf;
        float* dl = dbuf + (size_t)dims * HDC_MLP_FEATURES;
        if (cudaMemcpyAsync(dx, feat, sizeof(float) * dims * HDC_MLP_FEATURES, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            rc = HDC_ERR_CUDA;
        if (rc == HDC_OK) rc = hdc_mlp_forward(net, dx, dims, dl, st);
        if (rc == HDC_OK &&
            (cudaMemcpyAsync(logits.data(), dl, sizeof(float) * logits.size(), cudaMemcpyDeviceToHost, st) !=
                 cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = HDC_ERR_CUDA;
    }
    cudaFree(dbuf);
    hdc_mlp_destroy(net);
    return rc;
}

// k-th most likely valid tuple of axis i (outer axes within one column tile)
static int mlp_axis_choice(const std::vector<float>& logits, int dims, int i, const int64_t* L, const int64_t* M,
                           int dtype, int rank, hdc_tuple* t)
{
    const int nq = hdc_mlp_num_q_classes();
    const int64_t max_m = i < dims - 1 ? hdc_max_outer_fft_size(dtype) : 0;
    int rc = hdc_mlp_decode_axis(logits.data() + (size_t)i * (nq + 2), nq, L[i], M[i], dtype, max_m, rank, &t->m,
                                 &t->p, &t->q, &t->D);
    t->model_flops = model_flops_axis(L[i], t->m, t->q);
    t->ms = -1.0;
    return rc;
}

// Parameters from the learned predictor: its most likely class per axis, or
// (search) the fastest of its `topk` most likely classes per axis, timed
// one axis at a time with the others held (last axis first) on scratch
// buffers allocated here.
// Candidates of axis i for the guided search: the valid classes in
// decreasing score, the first topk of them, then the valid q-neighbours (one
// class down and one up) of the first two, at most 2 topk, distinct m.  The
// network locates the region; the neighbours cover a best q that sits
// between its top classes, as on axes longer than any it was trained on.
static std::vector<hdc_tuple> guided_candidates(const std::vector<float>& logits, int dims, int i, const int64_t* L,
                                                const int64_t* M, int dtype, int topk)
{
    const int nq = hdc_mlp_num_q_classes();
    const float* lg = logits.data() + (size_t)i * (nq + 2);
    const int one = lg[nq + 1] > lg[nq] ? 1 : 0;
    const int64_t max_m = i < dims - 1 ? hdc_max_outer_fft_size(dtype) : 0;
    std::vector<int> order(nq);
    for (int k = 0; k < nq; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lg[a] > lg[b]; });
    std::vector<hdc_tuple> out;
    std::vector<int> top;
    auto add = [&](int k) {
        if (k < 0 || k >= nq || (int)out.size() >= 2 * topk) return false;
        hdc_tuple c;
        if (hdc_mlp_decode_class(k, one, L[i], M[i], dtype, max_m, &c.m, &c.p, &c.q, &c.D) != HDC_OK) return false;
        for (const auto& o : out)
            if (o.m == c.m) return false;
        c.model_flops = model_flops_axis(L[i], c.m, c.q);
        c.ms = -1.0;
        out.push_back(c);
        return true;
    };
    for (int k : order) {
        if ((int)top.size() >= topk) break;
        if (add(k)) top.push_back(k);
    }
    for (size_t j = 0; j < top.size() && j < 2; ++j) {
        add(top[j] - 1);
        add(top[j] + 1);
    }
    return out;
}

static int predict_mlp(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch, const char* path,
                       cudaStream_t st, hdc_tuple* t, int topk, int64_t* timed)
{
    std::vector<float> logits;
    int rc = mlp_logits(dims, L, M, dtype, batch, path, st, logits);
    if (rc != HDC_OK) return rc;
    for (int i = 0; i < dims; ++i) {
        rc = mlp_axis_choice(logits, dims, i, L, M, dtype, 0, &t[i]);
        if (rc != HDC_OK) return rc;
    }
    if (topk <= 1) return HDC_OK;
    int64_t tot = batch;
    for (int i = 0; i < dims; ++i) tot *= L[i];
    const size_t esz = dtype == HDC_C128 ? 16 : 8;
    std::vector<hdc_tuple> cand[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) cand[i] = guided_candidates(logits, dims, i, L, M, dtype, topk);
    // the largest workspace of any combination the search can time
    size_t wsb = 0;
    int64_t idx[HDC_MAX_DIMS] = { 0, 0, 0 };
    while (true) {
        int64_t mm[HDC_MAX_DIMS], DD[HDC_MAX_DIMS];
        for (int j = 0; j < dims; ++j) {
            const hdc_tuple& c = cand[j].empty() ? t[j] : cand[j][idx[j]];
            mm[j] = c.m;
            DD[j] = c.D;
        }
        size_t b = 0;
        if (hdc_workspace_size(dims, L, M, mm, nullptr, nullptr, DD, dtype, batch, 0, &b) == HDC_OK)
            wsb = std::max(wsb, b);
        int k = dims - 1;
        while (k >= 0 && ++idx[k] >= (int64_t)std::max<size_t>(1, cand[k].size())) idx[k--] = 0;
        if (k < 0) break;
    }
    void *bf = nullptr, *bg = nullptr, *bh = nullptr, *bw = nullptr;
    if (cudaMalloc(&bf, tot * esz) != cudaSuccess || cudaMalloc(&bg, tot * esz) != cudaSuccess ||
        cudaMalloc(&bh, tot * esz) != cudaSuccess || cudaMalloc(&bw, wsb) != cudaSuccess) {
        cudaFree(bf); cudaFree(bg); cudaFree(bh); cudaFree(bw);
        return HDC_ERR_ALLOC;
    }
    cudaMemsetAsync(bf, 0, tot * esz, st);
    cudaMemsetAsync(bg, 0, tot * esz, st);
    for (int i = dims - 1; i >= 0; --i) {
        double best = -1.0;
        hdc_tuple pick = t[i];
        for (const auto& c : cand[i]) {
            hdc_tuple trial[HDC_MAX_DIMS];
            for (int j = 0; j < dims; ++j) trial[j] = t[j];
            trial[i] = c;
            const double ms = time_config(dims, bf, bg, bh, L, M, trial, dtype, batch, bw, wsb, 1, kPlanReps, st);
            if (timed) ++*timed;
            if (ms >= 0 && (best < 0 || ms < best)) { best = ms; pick = c; }
        }
        t[i] = pick;
        t[i].ms = best;
    }
    cudaStreamSynchronize(st);
    cudaFree(bf); cudaFree(bg); cudaFree(bh); cudaFree(bw);
    return HDC_OK;
}

HDC_EXPORT int hdc_plan_create(hdc_plan** out, int dims, const int64_t* L, const int64_t* M, const int64_t* m,
                               const int64_t* D, int dtype, int64_t batch, int mode, const char* tuning_db,
                               void* stream)
{
    if (!out || dims < 1 || dims > HDC_MAX_DIMS || !L || !M || batch < 1) return HDC_ERR_PARAM;
    if (dtype != HDC_C64 && dtype != HDC_C128) return HDC_ERR_DTYPE;
    hdc_plan pl;
    memset(&pl, 0, sizeof pl);
    pl.dims = dims;
    pl.dtype = dtype;
    pl.batch = batch;
    for (int i = 0; i < dims; ++i) { pl.L[i] = L[i]; pl.M[i] = M[i]; }
    const std::string key = db_key(dims, L, M, dtype, batch);
    if (mode == HDC_FIXED || mode == HDC_EXPLICIT) {
        for (int i = 0; i < dims; ++i) {
            int64_t mi = 0, p = 0, q = 0, Dv = 0;
            if (mode == HDC_EXPLICIT) {
                int rc = hdc_explicit_params(L[i], M[i], &mi, &p, &q);
                if (rc != HDC_OK) return rc;
            } else {
                if (!m) return HDC_ERR_PARAM;
                mi = m[i];
            }
            int rc = hdc_validate_axis(L[i], M[i], mi, 0, 0, D ? D[i] : 0, dtype, &p, &q, &Dv);
            if (rc != HDC_OK) return rc;
            pl.t[i].m = mi; pl.t[i].p = p; pl.t[i].q = q; pl.t[i].D = Dv;
            pl.t[i].model_flops = model_flops_axis(L[i], mi, q);
            pl.t[i].ms = -1.0;
        }
    } else if (mode == HDC_TUNE_EXHAUSTIVE || mode == HDC_TUNE_CACHED_ONLY) {
        if (!db_lookup(tuning_db, key, dims, pl.t)) {
            if (mode == HDC_TUNE_CACHED_ONLY) return HDC_ERR_NOT_TUNED;
            // tune on scratch buffers of the problem's shape (zeros suffice:
            // the kernels' work does not depend on the values)
            int64_t tot = batch;
            for (int i = 0; i < dims; ++i) tot *= L[i];
            const size_t esz = dtype == HDC_C128 ? 16 : 8;
            size_t wsb = 0;
            int rc = hdc_tune_workspace_size(dims, L, M, dtype, batch, kPlanRatio, kPlanMmin, &wsb);
            if (rc != HDC_OK) return rc;
            void *bf = nullptr, *bg = nullptr, *bh = nullptr, *bw = nullptr;
            cudaStream_t st = (cudaStream_t)stream;
            if (cudaMalloc(&bf, tot * esz) != cudaSuccess || cudaMalloc(&bg, tot * esz) != cudaSuccess ||
                cudaMalloc(&bh, tot * esz) != cudaSuccess || cudaMalloc(&bw, wsb) != cudaSuccess) {
                cudaFree(bf); cudaFree(bg); cudaFree(bh); cudaFree(bw);
                return HDC_ERR_ALLOC;
            }
            cudaMemsetAsync(bf, 0, tot * esz, st);
            cudaMemsetAsync(bg, 0, tot * esz, st);
            rc = hdc_tune_convnd(dims, L, M, dtype, batch, bf, bg, bh, bw, wsb, 1, kPlanReps, kPlanRatio, kPlanMmin, stream, pl.t, nullptr,
                                 0, &pl.timed);
            cudaStreamSynchronize(st);
            cudaFree(bf); cudaFree(bg); cudaFree(bh); cudaFree(bw);
            if (rc != HDC_OK) return rc;
            db_store(tuning_db, key, dims, pl.t);
        }
    } else if (mode == HDC_TUNE_RANDOM || mode == HDC_TUNE_PROXY) {
        const std::string k2 = key + (mode == HDC_TUNE_RANDOM ? " random" : " proxy");
        if (!db_lookup(tuning_db, k2, dims, pl.t)) {
            int64_t tot = batch;
            for (int i = 0; i < dims; ++i) tot *= L[i];
            const size_t esz = dtype == HDC_C128 ? 16 : 8;
            size_t wsb = 0;
            int rc = hdc_tune_workspace_size(dims, L, M, dtype, batch, kPlanRatio, kPlanMmin, &wsb);
            if (rc != HDC_OK) return rc;
            void *bf = nullptr, *bg = nullptr, *bh = nullptr, *bw = nullptr;
            cudaStream_t st = (cudaStream_t)stream;
            if (cudaMalloc(&bf, tot * esz) != cudaSuccess || cudaMalloc(&bg, tot * esz) != cudaSuccess ||
                cudaMalloc(&bh, tot * esz) != cudaSuccess || cudaMalloc(&bw, wsb) != cudaSuccess) {
                cudaFree(bf); cudaFree(bg); cudaFree(bh); cudaFree(bw);
                return HDC_ERR_ALLOC;
            }
            cudaMemsetAsync(bf, 0, tot * esz, st);
            cudaMemsetAsync(bg, 0, tot * esz, st);
            if (mode == HDC_TUNE_RANDOM)
                rc = hdc_tune_convnd_random(dims, L, M, dtype, batch, bf, bg, bh, bw, wsb, 1, kPlanReps, kPlanRatio, kPlanMmin,
                                            0, kPlanSeed, stream, pl.t, nullptr, 0, &pl.timed);
            else
                rc = hdc_tune_convnd_proxy(dims, L, M, dtype, batch, bf, bg, bh, bw, wsb, 1, kPlanReps, kPlanRatio, kPlanMmin,
                                           kPlanProxy, stream, pl.t, &pl.timed);
            cudaStreamSynchronize(st);
            cudaFree(bf); cudaFree(bg); cudaFree(bh); cudaFree(bw);
            if (rc != HDC_OK) return rc;
            db_store(tuning_db, k2, dims, pl.t);
        }
    } else if (mode == HDC_PREDICT_MLP || mode == HDC_PREDICT_MLP_SEARCH) {
        int rc = predict_mlp(dims, L, M, dtype, batch, tuning_db, (cudaStream_t)stream, pl.t,
                             mode == HDC_PREDICT_MLP_SEARCH ? 3 : 1, &pl.timed);
        if (rc != HDC_OK) return rc;
    } else {
        return HDC_ERR_PARAM;
    }
    int64_t mm[HDC_MAX_DIMS], pp[HDC_MAX_DIMS], qq[HDC_MAX_DIMS], DD[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) { mm[i] = pl.t[i].m; pp[i] = pl.t[i].p; qq[i] = pl.t[i].q; DD[i] = pl.t[i].D; }
    int rc = hdc_workspace_size(dims, L, M, mm, pp, qq, DD, dtype, batch, 1, &pl.ws);
    if (rc != HDC_OK) return rc;
    // the tables hdc_plan_execute reads are made here, so executing the plan
    // allocates nothing (and may be captured in a CUDA graph from the start);
    // on a host without a CUDA device the plan holds its parameters only
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
        rc = hdc_prepare(dims, L, M, mm, pp, qq, DD, dtype, batch);
        if (rc != HDC_OK) return rc;
    } else {
        cudaGetLastError();
    }
    hdc_plan* p = new (std::nothrow) hdc_plan(pl);
    if (!p) return HDC_ERR_ALLOC;
    *out = p;
    return HDC_OK;
}

HDC_EXPORT int hdc_plan_params(const hdc_plan* pl, int64_t* m, int64_t* p, int64_t* q, int64_t* D)
{
    if (!pl) return HDC_ERR_PARAM;
    for (int i = 0; i < pl->dims; ++i) {
        if (m) m[i] = pl->t[i].m;
        if (p) p[i] = pl->t[i].p;
        if (q) q[i] = pl->t[i].q;
        if (D) D[i] = pl->t[i].D;
    }
    return HDC_OK;
}

HDC_EXPORT size_t hdc_plan_workspace(const hdc_plan* pl) { return pl ? pl->ws : 0; }
HDC_EXPORT int64_t hdc_plan_timed(const hdc_plan* pl) { return pl ? pl->timed : -1; }

HDC_EXPORT int hdc_plan_execute(const hdc_plan* pl, const void* f, const void* g, void* h, void* ws,
                                size_t ws_bytes, void* stream)
{
    if (!pl) return HDC_ERR_PARAM;
    int64_t m[HDC_MAX_DIMS], p[HDC_MAX_DIMS], q[HDC_MAX_DIMS], D[HDC_MAX_DIMS];
    for (int i = 0; i < pl->dims; ++i) { m[i] = pl->t[i].m; p[i] = pl->t[i].p; q[i] = pl->t[i].q; D[i] = pl->t[i].D; }
    return hdc_convnd(pl->dims, f, g, h, pl->L, pl->M, m, p, q, D, (h == f || h == g) ? 1 : 0, pl->dtype, pl->batch,
                      ws, ws_bytes, stream);
}

HDC_EXPORT int hdc_plan_destroy(hdc_plan* pl)
{
    delete pl;
    return HDC_OK;
}

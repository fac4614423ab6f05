// hdc_batched.cu -- many independent 1-D convolutions of uneven length in one
// persistent launch.
//
// A batched plan turns n convolutions (lengths L_i, M_i = 2 L_i - 1, FFT
// sizes m_i chosen per size class) into four lists of work items, one per
// phase of the residue method:
//   phase 0  fold + m1-point FFTs of column tiles       (split convolutions)
//   phase 1  one residue of a whole row: fold, FFTs, product, inverse FFT
//            (fused convolutions), or one m2-point row of the split ones
//   phase 2  inverse m1-point FFTs of column tiles       (split convolutions)
//   phase 3  unfold of a chunk of one convolution's outputs (all)
// Every convolution's work lives in the same four phases, so one cooperative
// launch of as many blocks as fit on the GPU runs them all: blocks claim
// items of the current phase with an atomic counter, then meet at a grid
// barrier before the next phase.  The barrier's spin is bounded: when it
// runs out the block writes HDC_ERR_TIMEOUT into the status word of the
// workspace and returns (no trap, no hang); hdc_batched_status reads it.
// The launch (with the memset that clears the counters) can be captured in a
// CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "hdc.h"
#include "hdc_bodies.cuh"
#include "hdc_internal.h"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace hdc {

template <class V> struct BConv {
    TwTab<V> twN;
    const V* twm;  // packed stage tables of the m-point (fused) or m2-point (split rows) transform
    const V* twm1; // packed stage tables of the m1-point transform (split columns)
    const V* twml;  // the same two tables in scale-tangent form
    const V* twm1l;
    const V* tpm;   // split: zeta_m^{l1 c} at c m1 + l1 (column-major four-step twiddles)
    int64_t L, N, ws_off;
    int m, p, q, m1, m2, C, nct, per; // m1 == 0: fused; per = outputs per residue block
    FftPlan fpm;                      // plan of m (fused) or m2 (split rows)
    FftPlan fpm1;                     // plan of m1
};

struct BItem {
    int conv, a, b, c;
};

// One (convolution, residue) of a group of fused rows of one transform size
// (a phase-1 item with conv < 0: members [a, a + b) of the member list, m = c).
struct BMember {
    int conv, r;
};

// A group of k fused residue rows of one transform size m, as the k
// columns of one tile (element s of column j at s k + j): each column's fold
// (Eq. 1 inner sum and zeta_N^{r s}, its own convolution's inputs and
// parameters), the m-point FFTs of all columns at once, the products, the
// inverse FFT; column j's unscaled result to its residue's workspace row.
// A short transform alone would keep most of the block's threads idle at
// every stage (a 128-point FFT has 16 radix-8 butterflies); k of them fill it.
template <class V>
__device__ __forceinline__ void residue_rows_group(const BConv<V>* __restrict__ convs,
                                                   const BMember* __restrict__ mem, int k, int m,
                                                   const V* const* __restrict__ fp_, const V* const* __restrict__ gp_,
                                                   V* ws, V* smem, int tid, int nthr)
{
    const int n = k * m;
    V* sa = smem;
    V* sb = sa + smem_len<V>(n);
    V* sc = sb + smem_len<V>(n);
    for (int e = tid; e < n; e += nthr) {
        const int j = e / m, s = e - j * m;
        const BMember mb = mem[j];
        const BConv<V>& cv = convs[mb.conv];
        const V* fr = fp_[mb.conv];
        const V* gr = gp_[mb.conv];
        const int r = mb.r;
        V af = s < cv.L ? fr[s] : czero<V>(), ag = s < cv.L ? gr[s] : czero<V>();
        for (int t = 1; t < cv.p; ++t) {
            const int64_t jj = (int64_t)t * m + s;
            if (jj >= cv.L) break;
            if (r == 0) {
                af = cadd(af, fr[jj]);
                ag = cadd(ag, gr[jj]);
            } else {
                const V w = twn(cv.twN, (((int64_t)r * t) % cv.q) * m);
                af = cfma(fr[jj], w, af);
                ag = cfma(gr[jj], w, ag);
            }
        }
        if (r != 0) {
            const V w = twn(cv.twN, (int64_t)r * s);
            af = cmul(af, w);
            ag = cmul(ag, w);
        }
        sa[s * k + j] = af;
        sb[s * k + j] = ag;
    }
    __syncthreads();
    const BConv<V>& c0 = convs[mem[0].conv]; // every member has this m: same plan and tables
    fft_smem<V, false>(sa, sc, c0.fpm, k, k, 1, c0.twm, c0.twml, tid, nthr);
    fft_smem<V, false>(sb, sc, c0.fpm, k, k, 1, c0.twm, c0.twml, tid, nthr);
    for (int e = tid; e < n; e += nthr) sa[e] = cmul(sa[e], sb[e]);
    __syncthreads();
    fft_smem<V, true>(sa, sc, c0.fpm, k, k, 1, c0.twm, c0.twml, tid, nthr);
    for (int e = tid; e < n; e += nthr) {
        const int j = e / m, s = e - j * m;
        const BMember mb = mem[j];
        (ws + convs[mb.conv].ws_off + (int64_t)mb.r * m)[s] = sa[s * k + j];
    }
    __syncthreads();
}

// Workspace header (the first 256 bytes): phase counters, barrier, status,
// and the global-timer readings that split the launch into its phases: t[0]
// when block 0 starts, t[1..3] when block 0 leaves each grid barrier, t[4]
// when the last block ends.
struct BHeader {
    unsigned int ctr[4];
    unsigned int arrive;
    int status;
    unsigned long long t[5];
    unsigned int pad[48];
};
static_assert(sizeof(BHeader) == 256, "header must stay 256 bytes");

constexpr int kUnfoldChunk = 1024; // outputs per unfold item

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool grid_barrier(BHeader* hd, unsigned int target, long long spin_limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&hd->arrive, 1u);
        long long it = 0;
        int ok = 1;
        while (*(volatile unsigned int*)&hd->arrive < target) {
            if (*(volatile int*)&hd->status != 0 || ++it > spin_limit) {
                atomicCAS(&hd->status, 0, (int)HDC_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class V>
__global__ void __launch_bounds__(kMaxThreads)
k_batched(const BConv<V>* __restrict__ convs, const BItem* __restrict__ it0, const BItem* __restrict__ it1,
          const BItem* __restrict__ it2, const BItem* __restrict__ it3, const BMember* __restrict__ members,
          int n0, int n1, int n2, int n3,
          const V* const* __restrict__ fp_, const V* const* __restrict__ gp_, V* const* __restrict__ hp_, V* ws,
          BHeader* hd, long long spin_limit, int extra_arrivals)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    V* smem = reinterpret_cast<V*>(smraw);
    __shared__ int s_idx;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const BItem* lists[4] = { it0, it1, it2, it3 };
    if (blockIdx.x == 0 && tid == 0) hd->t[0] = global_ns();
    const int counts[4] = { n0, n1, n2, n3 };
    for (int ph = 0; ph < 4; ++ph) {
        const BItem* items = lists[ph];
        const int n = counts[ph];
        while (true) {
            if (tid == 0) s_idx = (int)atomicAdd(&hd->ctr[ph], 1u);
            __syncthreads();
            const int idx = s_idx;
            __syncthreads();
            if (idx >= n) break;
            const BItem itm = items[idx];
            if (ph == 1 && itm.conv < 0) {
                residue_rows_group<V>(convs, members + itm.a, itm.b, itm.c, fp_, gp_, ws, smem, tid, nthr);
                continue;
            }
            const BConv<V>& cv = convs[itm.conv];
            V* cws = ws + cv.ws_off;
            if (ph == 0) {
                // (conv, r, which, column tile): yf/yg [r][l1][c]
                const int r = itm.a, which = itm.b, ct = itm.c;
                const V* x = which ? gp_[itm.conv] : fp_[itm.conv];
                V* yb = cws + (int64_t)which * cv.q * cv.m + (int64_t)r * cv.m;
                fold_fft_cols_body<V>(x, yb, cv.m2, cv.m1, cv.p, cv.q, cv.N, cv.m2, 1, cv.L, r, (int64_t)ct * cv.C,
                                      cv.C, 1, cv.m2, cv.twN, cv.tpm, cv.twm1, cv.twm1l, cv.fpm1, smem, tid, nthr);
            } else if (ph == 1) {
                if (cv.m1 == 0) {
                    const int r = itm.a;
                    residue_row_body<V>(fp_[itm.conv], gp_[itm.conv], cws + (int64_t)r * cv.m, cv.L, cv.L, cv.m, cv.p,
                                        cv.q, r, cv.twN, cv.twm, cv.twml, cv.fpm, smem, tid, nthr);
                } else {
                    const int64_t row = itm.a;
                    V* yf = cws + row * cv.m2;
                    const V* yg = cws + (int64_t)cv.q * cv.m + row * cv.m2;
                    residue_row_body<V>(yf, yg, yf, cv.m2, cv.m2, cv.m2, 1, 1, 0, cv.twN, cv.twm, cv.twml, cv.fpm, smem, tid,
                                        nthr);
                }
            } else if (ph == 2) {
                const int r = itm.a, ct = itm.c;
                ifft_cols_body<V>(cws + (int64_t)r * cv.m, cv.m2, cv.m1, cv.q, cv.N, (int64_t)ct * cv.C, cv.C, 1,
                                  cv.twN, cv.tpm, cv.twm1, cv.twm1l, cv.fpm1, smem, tid, nthr);
            } else {
                const int64_t e0 = (int64_t)itm.a * kUnfoldChunk;
                const int64_t e1 = min((int64_t)cv.per, e0 + kUnfoldChunk);
                const int64_t Cn = cv.m1 ? cv.m2 : 1;
                const int64_t ma = cv.m1 ? cv.m1 : cv.m;
                const int64_t cs = cv.m1 ? cv.m2 : 1;
                const int64_t cc = cv.m1 ? 1 : 0;
                using T = typename real_of<V>::type;
                for (int64_t e = e0 + tid; e < e1; e += nthr) {
                    const int64_t i = div_idx(e, Cn), c = e - i * Cn;
                    unfold_elem<V, 4>(hp_[itm.conv], cws, cv.m, Cn, ma, i, c, cv.p, cv.q, cv.N, cs, cc, (int64_t)0,
                                      cv.L, 0, cv.q, 1, 1, (T)(1.0 / (double)cv.N), cv.twN);
                }
            }
        }
        if (ph < 3) {
            const unsigned int target = (unsigned int)(gridDim.x * (ph + 1)) + (unsigned int)extra_arrivals;
            if (!grid_barrier(hd, target, spin_limit)) return;
            if (blockIdx.x == 0 && tid == 0) hd->t[ph + 1] = global_ns();
        }
    }
    if (tid == 0) atomicMax(&hd->t[4], global_ns());
}

} // namespace hdc

using namespace hdc;

struct hdc_batched {
    int dtype;
    int64_t n;
    std::vector<int64_t> L, m, p, q, m1, m2;
    void* d_conv = nullptr;
    void* d_items[4] = { nullptr, nullptr, nullptr, nullptr };
    void* d_members = nullptr;
    int nitems[4] = { 0, 0, 0, 0 };
    size_t ws = 0;     // bytes, header included
    size_t smem = 0;   // dynamic shared memory of the launch
    int grid = 0;
    long long spin_limit = 1LL << 26;
    int extra_arrivals = 0;
};

namespace {

constexpr int64_t kBatchedSmem = 96 * 1024;

template <typename T> int64_t batched_col_elems() { return kBatchedSmem / (2 * (int64_t)sizeof(cx<T>)); }

// Route of one convolution in the batched kernel: fused when m fits one
// row tile; otherwise m = m1 m2 with the largest m2 <= max_row and
// m1 <= the column budget.  Returns false if neither fits.
template <typename T> bool batched_route(int64_t m, int64_t* m1, int64_t* m2)
{
    if (m <= max_row_fft<T>()) { *m1 = 0; *m2 = m; return true; }
    for (int64_t d = max_row_fft<T>(); d >= 2; --d)
        if (m % d == 0 && m / d <= batched_col_elems<T>()) { *m1 = m / d; *m2 = d; return true; }
    return false;
}

// Column tile of the batched kernel: as wide as the tile budget allows (up
// to 256 columns), since its blocks always have kMaxThreads threads: a short
// axis then still gives whole warps of butterflies.
template <typename T> int col_tile_b(int64_t Cn, int64_t ma)
{
    int64_t C = 256;
    while (C > 1 && ma * C > batched_col_elems<T>()) C >>= 1;
    while (C > 1 && C / 2 >= Cn) C >>= 1;
    return (int)C;
}

void free_plan(hdc_batched* b)
{
    if (!b) return;
    cudaFree(b->d_conv);
    cudaFree(b->d_members);
    for (auto& p : b->d_items) cudaFree(p);
    delete b;
}

template <typename T> int build(hdc_batched* b)
{
    using V = cx<T>;
    // creating a batched plan makes the twiddle tables its kernel reads
    TableScope tables(kTablesCreate);
    std::vector<BConv<V>> convs((size_t)b->n);
    std::vector<BItem> items[4];
    std::vector<std::pair<double, int64_t>> cost;
    int64_t off = 0;
    size_t smem = 0;
    b->m1.assign(b->n, 0);
    b->m2.assign(b->n, 0);
    for (int64_t i = 0; i < b->n; ++i) {
        BConv<V> cv;
        memset(&cv, 0, sizeof cv);
        int64_t m1 = 0, m2 = 0;
        if (!batched_route<T>(b->m[i], &m1, &m2)) return HDC_ERR_UNSUPPORTED_SIZE;
        cudaError_t e = cudaSuccess;
        cv.L = b->L[i];
        cv.m = (int)b->m[i];
        cv.p = (int)b->p[i];
        cv.q = (int)b->q[i];
        cv.N = b->q[i] * b->m[i];
        cv.m1 = (int)m1;
        cv.m2 = (int)m2;
        cv.twN = tw_table<T>(cv.N, &e);
        if (e != cudaSuccess) return HDC_ERR_CUDA;
        cv.twm = twiddles_fft<T>(m1 ? m2 : b->m[i], false, &e);
        if (e != cudaSuccess) return HDC_ERR_CUDA;
        cv.twml = twiddles_fft<T>(m1 ? m2 : b->m[i], true, &e);
        if (e != cudaSuccess) return HDC_ERR_CUDA;
        cv.fpm = fft_plan<T>(m1 ? m2 : b->m[i]);
        if (m1) {
            cv.twm1 = twiddles_fft<T>(m1, false, &e);
            if (e != cudaSuccess) return HDC_ERR_CUDA;
            cv.twm1l = twiddles_fft<T>(m1, true, &e);
            if (e != cudaSuccess) return HDC_ERR_CUDA;
            if (sizeof(T) == 8) {   // FP64 only, as in the one-pass kernels
                cv.tpm = twiddles_colmajor<T>(m1, m2, &e);
                if (e != cudaSuccess) return HDC_ERR_CUDA;
            }
            cv.fpm1 = fft_plan<T>(m1);
            cv.C = col_tile_b<T>(m2, m1);
            cv.nct = (int)((m2 + cv.C - 1) / cv.C);
        }
        cv.per = cv.m;
        cv.ws_off = off;
        off += ((m1 ? 2 : 1) * b->q[i] * b->m[i] + 31) / 32 * 32;
        b->m1[i] = m1;
        b->m2[i] = m2;
        convs[(size_t)i] = cv;
        smem = std::max(smem, (size_t)(3 * smem_len<V>(m1 ? m2 : b->m[i])) * sizeof(V));
        if (m1) smem = std::max(smem, (size_t)(2 * smem_len<V>(m1 * cv.C)) * sizeof(V));
        cost.emplace_back((double)cv.q * cv.m * std::log2((double)cv.m + 1.0) + (double)cv.q * cv.L, i);
    }
    // largest convolutions first in every phase: the tail of each phase is
    // made of small items
    std::sort(cost.begin(), cost.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    // fused residue rows of at most kGroupElems / 2 points are grouped by
    // size, kGroupElems / m rows to an item (the group's three tiles fit the
    // launch's shared memory)
    const int64_t kGroupElems = kBatchedSmem / (3 * (int64_t)sizeof(V));
    std::vector<BMember> members;
    std::vector<std::pair<double, BItem>> rows1;
    std::map<int, std::vector<BMember>> small;
    for (auto& ce : cost) {
        const int64_t i = ce.second;
        const BConv<V>& cv = convs[(size_t)i];
        const int ci = (int)i;
        const double rcost = (double)cv.m * std::log2((double)cv.m + 1.0) + (double)cv.L;
        if (cv.m1) {
            for (int r = 0; r < cv.q; ++r)
                for (int w = 0; w < 2; ++w)
                    for (int ct = 0; ct < cv.nct; ++ct) items[0].push_back({ ci, r, w, ct });
            for (int row = 0; row < cv.q * cv.m1; ++row)
                rows1.push_back({ (double)cv.m2 * std::log2((double)cv.m2 + 1.0), BItem{ ci, row, 0, 0 } });
            for (int r = 0; r < cv.q; ++r)
                for (int ct = 0; ct < cv.nct; ++ct) items[2].push_back({ ci, r, 0, ct });
        } else if (2 * (int64_t)cv.m <= kGroupElems) {
            for (int r = 0; r < cv.q; ++r) small[cv.m].push_back({ ci, r });
        } else {
            for (int r = 0; r < cv.q; ++r) rows1.push_back({ rcost, BItem{ ci, r, 0, 0 } });
        }
        const int nch = (cv.per + kUnfoldChunk - 1) / kUnfoldChunk;
        for (int k = 0; k < nch; ++k) items[3].push_back({ ci, k, 0, 0 });
    }
    for (auto& kv : small) {
        const int m = kv.first;
        const int kmax = (int)(kGroupElems / m);
        const auto& v = kv.second;
        for (size_t g0 = 0; g0 < v.size(); g0 += kmax) {
            const int k = (int)std::min<size_t>(kmax, v.size() - g0);
            BItem it{ -1, (int)members.size(), k, m };
            smem = std::max(smem, (size_t)(3 * smem_len<V>((int64_t)k * m)) * sizeof(V));
            double gc = 0.0;
            for (int j = 0; j < k; ++j) {
                members.push_back(v[g0 + j]);
                gc += (double)m * std::log2((double)m + 1.0) + (double)convs[(size_t)v[g0 + j].conv].L;
            }
            rows1.push_back({ gc, it });
        }
    }
    std::stable_sort(rows1.begin(), rows1.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (auto& ri : rows1) items[1].push_back(ri.second);
    if (!members.empty()) {
        if (cudaMalloc(&b->d_members, members.size() * sizeof(BMember)) != cudaSuccess) return HDC_ERR_ALLOC;
        if (cudaMemcpy(b->d_members, members.data(), members.size() * sizeof(BMember), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return HDC_ERR_CUDA;
    }
    if (cudaMalloc(&b->d_conv, convs.size() * sizeof(BConv<V>)) != cudaSuccess) return HDC_ERR_ALLOC;
    if (cudaMemcpy(b->d_conv, convs.data(), convs.size() * sizeof(BConv<V>), cudaMemcpyHostToDevice) != cudaSuccess)
        return HDC_ERR_CUDA;
    for (int ph = 0; ph < 4; ++ph) {
        b->nitems[ph] = (int)items[ph].size();
        if (items[ph].empty()) continue;
        if (cudaMalloc(&b->d_items[ph], items[ph].size() * sizeof(BItem)) != cudaSuccess) return HDC_ERR_ALLOC;
        if (cudaMemcpy(b->d_items[ph], items[ph].data(), items[ph].size() * sizeof(BItem), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return HDC_ERR_CUDA;
    }
    b->ws = sizeof(BHeader) + (size_t)off * sizeof(V) + 256;
    b->smem = std::max(smem, (size_t)1024);
    auto kern = k_batched<V>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess)
        return HDC_ERR_CUDA;
    int per_sm = 0, dev = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMaxThreads, b->smem) != cudaSuccess)
        return HDC_ERR_CUDA;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1 || nsm < 1) return HDC_ERR_UNSUPPORTED_SIZE;
    b->grid = per_sm * nsm;
    return HDC_OK;
}

template <typename T>
int launch(hdc_batched* b, const void* const* f, const void* const* g, void* const* h, void* ws, cudaStream_t st)
{
    using V = cx<T>;
    uintptr_t base = ((uintptr_t)ws + 255) & ~(uintptr_t)255;
    BHeader* hd = (BHeader*)base;
    V* data = (V*)(base + sizeof(BHeader));
    if (cudaMemsetAsync(hd, 0, sizeof(BHeader), st) != cudaSuccess) return HDC_ERR_CUDA;
    double flops = 0.0;
    for (int64_t i = 0; i < b->n; ++i) {
        const double md = (double)b->m[i];
        flops += (double)b->q[i] * (15.0 * md * std::log2(md > 1 ? md : 2) + 6.0 * md + 24.0 * b->L[i]) +
                 2.0 * b->L[i];
    }
    LaunchScope ls(K_BATCHED, st, flops, 0.0);
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3(kMaxThreads);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const BConv<V>* cv = (const BConv<V>*)b->d_conv;
    const BItem* i0 = (const BItem*)b->d_items[0];
    const BItem* i1 = (const BItem*)b->d_items[1];
    const BItem* i2 = (const BItem*)b->d_items[2];
    const BItem* i3 = (const BItem*)b->d_items[3];
    const BMember* mem = (const BMember*)b->d_members;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_batched<V>, cv, i0, i1, i2, i3, mem, b->nitems[0], b->nitems[1],
                                       b->nitems[2], b->nitems[3], (const V* const*)f, (const V* const*)g,
                                       (V* const*)h, data, hd, b->spin_limit, b->extra_arrivals);
    return e == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}

} // namespace

HDC_EXPORT int hdc_batched_create(hdc_batched** out, int64_t n, const int64_t* L, const int64_t* m, int dtype)
{
    if (!out || n < 1 || !L || !m) return HDC_ERR_PARAM;
    if (dtype != HDC_C64 && dtype != HDC_C128) return HDC_ERR_DTYPE;
    hdc_batched* b = new (std::nothrow) hdc_batched;
    if (!b) return HDC_ERR_ALLOC;
    b->dtype = dtype;
    b->n = n;
    b->L.assign(L, L + n);
    b->m.assign(m, m + n);
    b->p.resize(n);
    b->q.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t Dv = 0;
        int rc = hdc_validate_axis(L[i], 2 * L[i] - 1, m[i], 0, 0, 0, dtype, &b->p[i], &b->q[i], &Dv);
        if (rc != HDC_OK) { free_plan(b); return rc; }
    }
    int rc = dtype == HDC_C128 ? build<double>(b) : build<float>(b);
    if (rc != HDC_OK) { free_plan(b); return rc; }
    *out = b;
    return HDC_OK;
}

HDC_EXPORT size_t hdc_batched_workspace(const hdc_batched* b) { return b ? b->ws : 0; }

HDC_EXPORT int hdc_batched_params(const hdc_batched* b, int64_t* m, int64_t* p, int64_t* q, int64_t* m1, int64_t* m2)
{
    if (!b) return HDC_ERR_PARAM;
    for (int64_t i = 0; i < b->n; ++i) {
        if (m) m[i] = b->m[i];
        if (p) p[i] = b->p[i];
        if (q) q[i] = b->q[i];
        if (m1) m1[i] = b->m1[i];
        if (m2) m2[i] = b->m2[i];
    }
    return HDC_OK;
}

HDC_EXPORT int hdc_batched_execute(hdc_batched* b, const void* const* f, const void* const* g, void* const* h,
                                   void* workspace, size_t ws_bytes, void* stream)
{
    if (!b || !f || !g || !h) return HDC_ERR_PARAM;
    if (!workspace || ws_bytes < b->ws) return HDC_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    return b->dtype == HDC_C128 ? launch<double>(b, f, g, h, workspace, st) : launch<float>(b, f, g, h, workspace, st);
}

HDC_EXPORT int hdc_batched_status(const void* workspace, int* status)
{
    if (!workspace || !status) return HDC_ERR_PARAM;
    uintptr_t base = ((uintptr_t)workspace + 255) & ~(uintptr_t)255;
    int v = 0;
    if (cudaMemcpy(&v, (const void*)(base + offsetof(BHeader, status)), sizeof v, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return HDC_ERR_CUDA;
    *status = v;
    return HDC_OK;
}

HDC_EXPORT int hdc_batched_phase_ms(const void* workspace, double* ms)
{
    if (!workspace || !ms) return HDC_ERR_PARAM;
    uintptr_t base = ((uintptr_t)workspace + 255) & ~(uintptr_t)255;
    unsigned long long t[5];
    if (cudaMemcpy(t, (const void*)(base + offsetof(BHeader, t)), sizeof t, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HDC_ERR_CUDA;
    for (int i = 0; i < 4; ++i) ms[i] = t[i + 1] >= t[i] ? (double)(t[i + 1] - t[i]) * 1e-6 : 0.0;
    return HDC_OK;
}

HDC_EXPORT int hdc_batched_set_barrier(hdc_batched* b, long long spin_limit, int extra_arrivals)
{
    if (!b || spin_limit < 1 || extra_arrivals < 0) return HDC_ERR_PARAM;
    b->spin_limit = spin_limit;
    b->extra_arrivals = extra_arrivals;
    return HDC_OK;
}

HDC_EXPORT int hdc_batched_destroy(hdc_batched* b)
{
    free_plan(b);
    return HDC_OK;
}

// ------------------------------------------------------------- tuning

namespace {

// Size class of a length: floor(log2 L).
int size_class(int64_t L)
{
    int k = 0;
    while ((L >> (k + 1)) > 0) ++k;
    return k;
}

template <typename T> bool batched_ok(int64_t m)
{
    int64_t a = 0, b = 0;
    return batched_route<T>(m, &a, &b);
}

} // namespace

HDC_EXPORT int hdc_batched_tune(int64_t n, const int64_t* L, int dtype, const void* const* f_host,
                                const void* const* g_host, void* const* h_host, int reps, int max_cands,
                                void* stream, int64_t* m_out, double* ms_out)
{
    if (n < 1 || !L || !f_host || !g_host || !h_host || !m_out || reps < 1 || max_cands < 1) return HDC_ERR_PARAM;
    if (dtype != HDC_C64 && dtype != HDC_C128) return HDC_ERR_DTYPE;
    cudaStream_t st = (cudaStream_t)stream;
    // A class's schedule is its residue count q and a size rule: every member
    // gets its own m >= ceil(M_i / q), either the next 2^a 3^b 5^c 7^d (the
    // least padding), the next 2^a or 3 2^a (more padding, but transforms
    // of radix-8, -4 and -2 stages and at most one radix-3 one, which cost
    // fewer FP64 instructions per point than radix 3, 5 and 7), or the next
    // 2^a, 3 2^a or 5 2^a (in between), so the FFT size follows each length.
    // A schedule is encoded as 3 q + rule.
    static const int64_t qs[] = { 1, 2, 3, 4, 5, 6, 8, 10, 12, 16 };
    auto m_for = [&](int64_t Li, int64_t sched) -> int64_t {
        const int64_t q = sched / 3;
        const int rule = (int)(sched % 3);
        const int64_t M = 2 * Li - 1;
        const int64_t lo = (M + q - 1) / q;
        int64_t m = hdc_next_good_size(lo);
        if (rule != 0) {
            int64_t p2 = 1;
            while (p2 < lo) p2 *= 2;
            int64_t t3 = 3;
            while (t3 < lo) t3 *= 2;
            m = std::min(p2, t3);
            if (rule == 2) {
                int64_t t5 = 5;
                while (t5 < lo) t5 *= 2;
                m = std::min(m, t5);
            }
        }
        if (m < 1) return -1;
        const bool ok = dtype == HDC_C128 ? batched_ok<double>(m) : batched_ok<float>(m);
        return ok ? m : -1;
    };
    std::vector<std::vector<int64_t>> members(64);
    for (int64_t i = 0; i < n; ++i) {
        if (L[i] < 1) return HDC_ERR_PARAM;
        members[size_class(L[i])].push_back(i);
    }
    std::vector<int> order;
    std::vector<std::vector<int64_t>> cands(64);
    std::vector<double> work(64, 0.0);
    for (int k = 0; k < 64; ++k) {
        if (members[k].empty()) continue;
        int64_t Lmin = INT64_MAX;
        for (int64_t i : members[k]) { Lmin = std::min(Lmin, L[i]); work[k] += (double)L[i]; }
        for (int64_t q : qs) {
            if ((int64_t)cands[k].size() >= max_cands) break;
            // q is usable when every member has an m >= 16 that the kernel supports
            if (!((2 * Lmin - 1 + q - 1) / q >= 16 || q == 1)) continue;
            for (int rule = 0; rule < 3 && (int64_t)cands[k].size() < max_cands; ++rule) {
                // usable when every member gets a supported m; skipped when
                // every member gets the m of the rule before (nothing new)
                bool ok = true, same = rule > 0;
                for (int64_t i : members[k]) {
                    const int64_t mi = m_for(L[i], 3 * q + rule);
                    ok = ok && mi > 0;
                    same = same && mi == m_for(L[i], 3 * q + rule - 1);
                }
                if (ok && !same) cands[k].push_back(3 * q + rule);
            }
        }
        if (cands[k].empty()) return HDC_ERR_UNSUPPORTED_SIZE;
        for (int64_t i : members[k]) m_out[i] = m_for(L[i], cands[k][0]);
        order.push_back(k);
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    void* dptr = nullptr;
    if (cudaMalloc(&dptr, 3 * (size_t)n * sizeof(void*)) != cudaSuccess) return HDC_ERR_ALLOC;
    const void** pf = (const void**)dptr;
    const void** pg = pf + n;
    void** ph = (void**)(pg + n);
    cudaMemcpy(pf, f_host, n * sizeof(void*), cudaMemcpyHostToDevice);
    cudaMemcpy(pg, g_host, n * sizeof(void*), cudaMemcpyHostToDevice);
    cudaMemcpy(ph, h_host, n * sizeof(void*), cudaMemcpyHostToDevice);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    void* ws = nullptr;
    size_t ws_cap = 0;
    int rc = HDC_OK;
    // time the whole batch with the current assignment (median of reps)
    auto time_all = [&](double* out) -> int {
        hdc_batched* b = nullptr;
        int r = hdc_batched_create(&b, n, L, m_out, dtype);
        if (r != HDC_OK) return r;
        if (b->ws > ws_cap) {
            cudaFree(ws);
            ws = nullptr;
            ws_cap = 0;
            if (cudaMalloc(&ws, b->ws) != cudaSuccess) { hdc_batched_destroy(b); return HDC_ERR_ALLOC; }
            ws_cap = b->ws;
        }
        hdc_batched_execute(b, pf, pg, ph, ws, ws_cap, st);
        std::vector<float> ts;
        for (int k = 0; k < reps; ++k) {
            cudaEventRecord(e0, st);
            hdc_batched_execute(b, pf, pg, ph, ws, ws_cap, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ts.push_back(t);
        }
        int stt = 0;
        hdc_batched_status(ws, &stt);
        hdc_batched_destroy(b);
        if (stt != 0) return stt;
        std::sort(ts.begin(), ts.end());
        *out = ts[ts.size() / 2];
        return HDC_OK;
    };
    double best = 0.0;
    rc = time_all(&best);
    // one class at a time, largest work first, the others held (Section 4.2)
    for (int k : order) {
        if (rc != HDC_OK) break;
        int64_t bestq = cands[k][0];
        for (size_t c = 1; c < cands[k].size(); ++c) {
            for (int64_t i : members[k]) m_out[i] = m_for(L[i], cands[k][c]);
            double t = 0.0;
            const int r = time_all(&t);
            if (r == HDC_OK && t < best) { best = t; bestq = cands[k][c]; }
        }
        for (int64_t i : members[k]) m_out[i] = m_for(L[i], bestq);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ws);
    cudaFree(dptr);
    if (ms_out) *ms_out = best;
    return rc;
}

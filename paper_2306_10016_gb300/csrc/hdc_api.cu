// hdc_api.cu -- host side of the C ABI declared in include/hdc.h:
// parameter derivation and validation (Section 2.5), the twiddle-table cache,
// workspace sizing, and the drivers that sequence the kernels of
// hdc_kernels.cu for 1-D rows and the N-D recursion over axes (Section 3.6).
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <stdint.h>
#include <string.h>
#include <tuple>

#include "hdc.h"
#include "hdc_internal.h"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace hdc {

// The CUDA error behind the last HDC_ERR_CUDA of a convolution call
// (hdc_last_cuda_error).
static std::atomic<int> g_last_cuda_error{ 0 };

static int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return HDC_OK;
    if (tables_missing()) {
        tables_missing() = false;
        return HDC_ERR_NOT_PREPARED;
    }
    g_last_cuda_error.store((int)e);
    return HDC_ERR_CUDA;
}

template <typename T> cudaError_t launch_twiddle(cx<T>* tw, int64_t n, cudaStream_t st);
template <typename T> cudaError_t launch_twiddle_lf(cx<T>* tw, int64_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_twiddle_strided(cx<T>* tw, int64_t count, int64_t N, int64_t stride, cudaStream_t st);
template <typename T> cudaError_t launch_twiddle_colmajor(cx<T>* tw, int64_t ma, int64_t Cn, cudaStream_t st);

// ----------------------------------------------------------- FFT plans

FftPlan make_fft_plan(int64_t n, bool r16, bool r2)
{
    FftPlan fp;
    memset(&fp, 0, sizeof(fp));
    fp.n = (int)n;
    int64_t k = n;
    int ns = 0;
    if (r2) {
        // latency plan: radix 2 throughout the power-of-two part
        while (k % 2 == 0 && ns < HDC_MAX_STAGES) { fp.rad[ns++] = 2; k /= 2; }
    } else if (r16) {
        // radix-16 stages only where they save a stage over radix 8 on the
        // power-of-two part 2^e: ceil(e / 4) < ceil(e / 3)
        int e = 0;
        for (int64_t t = n; t % 2 == 0; t /= 2) ++e;
        if ((e + 3) / 4 < (e + 2) / 3)
            while (k % 16 == 0 && ns < HDC_MAX_STAGES) { fp.rad[ns++] = 16; k /= 16; }
    }
    while (k % 8 == 0 && ns < HDC_MAX_STAGES) { fp.rad[ns++] = 8; k /= 8; }
    while (k % 4 == 0 && ns < HDC_MAX_STAGES) { fp.rad[ns++] = 4; k /= 4; }
    while (k % 2 == 0 && ns < HDC_MAX_STAGES) { fp.rad[ns++] = 2; k /= 2; }
    while (k % 7 == 0 && ns < HDC_MAX_STAGES) { fp.rad[ns++] = 7; k /= 7; }
    while (k % 5 == 0 && ns < HDC_MAX_STAGES) { fp.rad[ns++] = 5; k /= 5; }
    while (k % 3 == 0 && ns < HDC_MAX_STAGES) { fp.rad[ns++] = 3; k /= 3; }
    fp.nst = ns;
    // packed twiddle table: a sub-table of Ns R entries per stage after the
    // first
    int64_t ns_done = 1, off = 0;
    for (int s = 0; s < ns; ++s) {
        fp.toff[s] = (int32_t)off;
        if (ns_done > 1) off += ns_done * fp.rad[s];
        ns_done *= fp.rad[s];
    }
    fp.tlen = (int32_t)(off > 0 ? off : 1);
    return fp;
}

// ------------------------------------------------------- twiddle cache

namespace {
std::mutex g_tw_mu;
std::map<std::tuple<int, int64_t, int>, void*> g_tw;
thread_local int t_table_mode = kTablesLookup;
thread_local bool t_tables_missing = false;
} // namespace

TableScope::TableScope(int mode) : saved(t_table_mode) { t_table_mode = mode; }
TableScope::~TableScope() { t_table_mode = saved; }
int table_mode() { return t_table_mode; }
bool& tables_missing() { return t_tables_missing; }

// The cached table under (current device, n, kind), made by `fill` (a
// launcher writing `count` elements of `esz` bytes on the given stream) when
// it is missing and the thread's table mode allows it.  A new table is
// built on a private stream and waited for, so it is complete before any
// stream of the caller can read it.  In lookup mode a missing table sets
// tables_missing() and fails (cudaErrorInvalidResourceHandle).
template <class Fill>
static void* cached_table(int64_t n, int kind, size_t bytes, Fill fill, cudaError_t* err)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *err = e; return nullptr; }
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto key = std::make_tuple(dev, n, kind);
    auto it = g_tw.find(key);
    if (it != g_tw.end()) return it->second;
    if (t_table_mode == kTablesLookup) {
        t_tables_missing = true;
        *err = cudaErrorInvalidResourceHandle;
        return nullptr;
    }
    void* p = nullptr;
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) { *err = e; return nullptr; }
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        e = fill(p, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(s);
    }
    if (e != cudaSuccess) { cudaFree(p); *err = e; return nullptr; }
    g_tw[key] = p;
    return p;
}

// A 256 MiB device buffer per device that the tuners overwrite before each
// timed replay to evict the 129 MB L2 (kept with the tables, freed by
// hdc_release_caches); null if it cannot be made.
void* tuning_flush_buffer(size_t* bytes)
{
    constexpr size_t kFlush = (size_t)256 << 20;
    cudaError_t e = cudaSuccess;
    void* p = cached_table(
        (int64_t)kFlush, -2, kFlush, [&](void* q, cudaStream_t s) { return cudaMemsetAsync(q, 0, kFlush, s); }, &e);
    *bytes = kFlush;
    return p;
}

template <typename T> static const cx<T>* twiddle_table(int64_t n, bool lf, cudaError_t* err)
{
    const int kind = (sizeof(T) == 8 ? 1 : 0) + (lf ? 2 : 0);
    return reinterpret_cast<const cx<T>*>(cached_table(
        n, kind, (size_t)n * sizeof(cx<T>),
        [&](void* p, cudaStream_t s) {
            return lf ? launch_twiddle_lf<T>(reinterpret_cast<cx<T>*>(p), n, s)
                      : launch_twiddle<T>(reinterpret_cast<cx<T>*>(p), n, s);
        },
        err));
}

// Packed per-stage twiddle tables of the n-point transform (FftPlan), plain
// or twiddle-merged form; cached like the full tables.
template <typename T> const cx<T>* twiddles_fft(int64_t n, bool lf, cudaError_t* err, bool r16ok)
{
    return twiddles_fft_plan<T>(fft_plan<T>(n, r16ok), lf, err);
}
template const cx<double>* twiddles_fft<double>(int64_t, bool, cudaError_t*, bool);
template const cx<float>* twiddles_fft<float>(int64_t, bool, cudaError_t*, bool);

template <typename T> const cx<T>* twiddles_fft_plan(const FftPlan& fp, bool lf, cudaError_t* err)
{
    // the plans of one size differ in their first radices (16, 8 or 2), which
    // the key tells apart
    const int64_t n = fp.n;
    const int first = fp.nst > 0 ? fp.rad[0] : 0;
    const int kind = (sizeof(T) == 8 ? 1 : 0) + (lf ? 2 : 0) + 4 + (first == 16 ? 8 : 0) +
                     (first == 2 && n % 4 == 0 && fp.nst > 1 && fp.rad[1] == 2 ? 16 : 0);
    return reinterpret_cast<const cx<T>*>(cached_table(
        n, kind, (size_t)fp.tlen * sizeof(cx<T>),
        [&](void* p, cudaStream_t s) { return launch_twiddle_fft_into<T>(reinterpret_cast<cx<T>*>(p), fp, lf, s); },
        err));
}
template const cx<double>* twiddles_fft_plan<double>(const FftPlan&, bool, cudaError_t*);
template const cx<float>* twiddles_fft_plan<float>(const FftPlan&, bool, cudaError_t*);

// An FP32 fold/unfold table of N entries is kept whole up to this size; a
// larger one is two tables of about sqrt(N) entries (TwTab).
constexpr int64_t kTwFullMax = (int64_t)1 << 16;

template <typename T> static const cx<T>* strided_table(int64_t count, int64_t N, int64_t stride, int kind,
                                                        cudaError_t* err)
{
    // kinds 8 / 16 + dtype: the lo / hi table of N; the key's size field is N
    return reinterpret_cast<const cx<T>*>(cached_table(
        N, (sizeof(T) == 8 ? 1 : 0) + kind, (size_t)count * sizeof(cx<T>),
        [&](void* p, cudaStream_t s) {
            return launch_twiddle_strided<T>(reinterpret_cast<cx<T>*>(p), count, N, stride, s);
        },
        err));
}

template <typename T> TwTab<cx<T>> tw_table(int64_t N, cudaError_t* err)
{
    TwTab<cx<T>> t{ nullptr, nullptr, nullptr, 0 };
    // FP64 keeps one table: its kernels are bound by FP64 arithmetic, which
    // the extra complex product would add to
    if (sizeof(T) == 8 || N <= kTwFullMax) {
        t.full = twiddle_table<T>(N, false, err);
        return t;
    }
    int lb = 0;
    while (((int64_t)1 << (2 * lb)) < N) ++lb;
    const int64_t S = (int64_t)1 << lb;
    t.lb = lb;
    t.lo = strided_table<T>(S, N, 1, 8, err);
    if (!t.lo) return t;
    t.hi = strided_table<T>((N + S - 1) / S, N, S, 16, err);
    return t;
}
// The column-major four-step twiddles of an ma x Cn split (cached per pair).
template <typename T> const cx<T>* twiddles_colmajor(int64_t ma, int64_t Cn, cudaError_t* err)
{
    // kind 32 + dtype, with ma folded into the kind so the key is (ma, Cn)
    return reinterpret_cast<const cx<T>*>(cached_table(
        Cn, (sizeof(T) == 8 ? 1 : 0) + 32 + (int)ma * 64, (size_t)(ma * Cn) * sizeof(cx<T>),
        [&](void* p, cudaStream_t s) { return launch_twiddle_colmajor<T>(reinterpret_cast<cx<T>*>(p), ma, Cn, s); },
        err));
}
template const cx<double>* twiddles_colmajor<double>(int64_t, int64_t, cudaError_t*);
template const cx<float>* twiddles_colmajor<float>(int64_t, int64_t, cudaError_t*);

template TwTab<cx<double>> tw_table<double>(int64_t, cudaError_t*);
template TwTab<cx<float>> tw_table<float>(int64_t, cudaError_t*);

template <typename T> const cx<T>* twiddles(int64_t n, cudaError_t* err) { return twiddle_table<T>(n, false, err); }
template const cx<double>* twiddles<double>(int64_t, cudaError_t*);
template const cx<float>* twiddles<float>(int64_t, cudaError_t*);

// ----------------------------------------------------------- axis plan

// One axis.  The loop runs over the q residues of g, transformed at m
// points; f is transformed at mf = m / lam points with lam q residues
// (residue matching, Section 3.5).  Equal lengths: Lf = L, mf = m, pf = p,
// lam = 1.
struct Axis {
    int64_t L, M, m, p, q, D, N; // g: length, padded length, FFT size, fold blocks, residues, per pass, N = q m
    int64_t Lf, mf, pf, lam;     // f: length, FFT size, fold blocks; lam = m / mf
    int64_t m1, m2;              // m1 < 0: m not supported (no split within the tile limits)
    int dtype;
    int64_t o, Lw, pout; // output window [o, o + Lw) of the linear convolution; pout = ceil((o + Lw) / m)
};

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static bool good_size(int64_t n)
{
    if (n < 1) return false;
    for (int f : { 2, 3, 5, 7 })
        while (n % f == 0) n /= f;
    return n == 1;
}

// Split m = m1 m2 admissible: m2 <= max_row, m1 <= max_col, and lam | m1
// (f's transform then splits as (m1 / lam) m2 with the same rows).
template <typename T> static bool split_ok(int64_t m, int64_t d, int64_t lam)
{
    return m % d == 0 && m / d <= max_col_fft<T>() && (m / d) % lam == 0;
}

template <typename T> static bool splittable(int64_t m, int64_t lam)
{
    for (int64_t d = max_row_fft<T>(); d >= 2; --d)
        if (split_ok<T>(m, d, lam)) return true;
    return false;
}

template <typename T> static void split_m(Axis& a)
{
    a.m1 = 0;
    a.m2 = a.m;
    if (a.m <= max_row_fft<T>()) return;
    if (!splittable<T>(a.m, a.lam)) a.m1 = -1; // unsupported
}

static int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 152;
    }
    return n;
}

// Route of one 1-D pass over B rows: fused residue kernel (m1 = 0) or the
// split m = m1 m2.  FP64 work runs at a few flops per clock per SM, so the
// choice is made for parallelism: keep the fused kernel when it already
// launches two blocks per SM (or m is too small to split usefully);
// otherwise take the largest row length m2 whose middle pass has two blocks
// per SM, else the split with the most rows.
template <typename T> static void route_for(const Axis& a, int64_t B, int64_t* m1o, int64_t* m2o)
{
    const int64_t Dg = a.D < a.q ? a.D : a.q;
    const int64_t want = 2 * (int64_t)sm_count();
    const bool fused_ok = a.m <= max_row_fft<T>();
    if (fused_ok && (B * Dg >= want || a.m < 512)) { *m1o = 0; *m2o = a.m; return; }
    int64_t b1 = -1, b2 = -1;
    const int64_t top = a.m / 2 < max_row_fft<T>() ? a.m / 2 : max_row_fft<T>();
    for (int64_t d = top; d >= 32; --d) {
        if (a.m % d) continue;
        const int64_t m1 = a.m / d;
        if (m1 > max_col_fft<T>()) break;
        if (m1 % a.lam) continue;
        b1 = m1; b2 = d;
        if (Dg * B * m1 >= want) break;
    }
    if (b1 < 0 || (fused_ok && Dg * B * b1 < 4 * B * Dg)) {
        if (fused_ok) { *m1o = 0; *m2o = a.m; return; }
        // no split down to rows of 32: the largest admissible m2
        for (int64_t d = max_row_fft<T>(); d >= 2; --d)
            if (split_ok<T>(a.m, d, a.lam)) { b1 = a.m / d; b2 = d; break; }
    }
    *m1o = b1; *m2o = b2;
}

static void route(const Axis& a, int64_t B, int dtype, int64_t* m1, int64_t* m2)
{
    if (dtype == HDC_C128) route_for<double>(a, B, m1, m2);
    else route_for<float>(a, B, m1, m2);
}

// the largest split m1 m2 within the row and column tile limits (2^23 in
// FP64, 2^25 in FP32); an m of that size whose factors do not fit both
// limits is still rejected when the axis is resolved
static int64_t max_fft(int dtype)
{
    return dtype == HDC_C128 ? max_row_fft<double>() * max_col_fft<double>()
                             : max_row_fft<float>() * max_col_fft<float>();
}
static int64_t max_padded(int dtype) { return dtype == HDC_C128 ? (int64_t)1 << 25 : (int64_t)1 << 26; }

// One axis.  The output window [o, o + Lw) of the full linear convolution
// (length 2L - 1) is alias-free when the padded length reaches past every
// output that could wrap onto the window: M >= 2L - 1 - o (o = 0, Lw = L is
// the first-L convolution of Eq. 4 and needs M >= 2L - 1, Section 3.1).
static int resolve_axis(int64_t L, int64_t M, int64_t m, int64_t p, int64_t q, int64_t D, int dtype, Axis* out,
                        int64_t o = 0, int64_t Lw = -1)
{
    if (dtype != HDC_C64 && dtype != HDC_C128) return HDC_ERR_DTYPE;
    if (Lw < 0) Lw = L;
    if (L < 1 || M < 1 || m < 1 || p < 0 || q < 0 || D < 0 || o < 0 || Lw < 1) return HDC_ERR_PARAM;
    if (o + Lw > 2 * L - 1) return HDC_ERR_PARAM;
    if (M < 2 * L - 1 - o) return HDC_ERR_ALIAS;
    if (p == 0) p = ceil_div(L, m);
    if (q == 0) q = ceil_div(M, m);
    if (p * m < L || q * m < M) return HDC_ERR_PARAM;
    if (o + Lw > q * m) return HDC_ERR_ALIAS;
    if (D == 0) D = q;
    if (D > q) return HDC_ERR_PARAM;
    if (!good_size(m) || m > max_fft(dtype)) return HDC_ERR_UNSUPPORTED_SIZE;
    if (q > max_padded(dtype) / m) return HDC_ERR_UNSUPPORTED_SIZE;
    Axis a;
    a.L = L; a.M = M; a.m = m; a.p = p; a.q = q; a.D = D; a.N = q * m;
    a.Lf = L; a.mf = m; a.pf = p; a.lam = 1;
    a.dtype = dtype;
    a.o = o; a.Lw = Lw; a.pout = ceil_div(o + Lw, m);
    if (dtype == HDC_C128) split_m<double>(a); else split_m<float>(a);
    if (a.m1 < 0) return HDC_ERR_UNSUPPORTED_SIZE;
    if (out) *out = a;
    return HDC_OK;
}

// One axis with unequal lengths (Section 3.5): f of length Lf transformed at
// mf points, g of length Lg at mg = lam mf points; pf = ceil(Lf / mf),
// pg = ceil(Lg / mg), qg = ceil(M / mg), qf = lam qg, N = qg mg = qf mf.  The
// window [o, o + Lw) of the linear convolution (length Lf + Lg - 1) is
// alias-free when M >= Lf + Lg - 1 - o and o + Lw <= N.
static int resolve_axis_uneq(int64_t Lf, int64_t Lg, int64_t M, int64_t mf, int64_t lam, int64_t D, int dtype,
                             Axis* out, int64_t o, int64_t Lw)
{
    if (dtype != HDC_C64 && dtype != HDC_C128) return HDC_ERR_DTYPE;
    if (Lw < 0) Lw = Lg;
    if (Lf < 1 || Lg < 1 || mf < 1 || lam < 1 || D < 0 || o < 0 || Lw < 1) return HDC_ERR_PARAM;
    if (M <= 0) M = Lf + Lg - 1 - o;
    if (o + Lw > Lf + Lg - 1) return HDC_ERR_PARAM;
    if (M < Lf + Lg - 1 - o) return HDC_ERR_ALIAS;
    const int64_t mg = mf * lam;
    if (!good_size(mf) || !good_size(mg) || mg > max_fft(dtype)) return HDC_ERR_UNSUPPORTED_SIZE;
    const int64_t qg = ceil_div(M, mg);
    if (qg * lam > max_padded(dtype) / mf) return HDC_ERR_UNSUPPORTED_SIZE;
    if (o + Lw > qg * mg) return HDC_ERR_ALIAS;
    if (D == 0) D = qg;
    if (D > qg) return HDC_ERR_PARAM;
    Axis a;
    a.L = Lg; a.M = M; a.m = mg; a.p = ceil_div(Lg, mg); a.q = qg; a.D = D; a.N = qg * mg;
    a.Lf = Lf; a.mf = mf; a.pf = ceil_div(Lf, mf); a.lam = lam;
    a.dtype = dtype;
    a.o = o; a.Lw = Lw; a.pout = ceil_div(o + Lw, mg);
    if (dtype == HDC_C128) split_m<double>(a); else split_m<float>(a);
    if (a.m1 < 0) return HDC_ERR_UNSUPPORTED_SIZE;
    if (out) *out = a;
    return HDC_OK;
}

// ------------------------------------------------------------ workspace

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Elements (complex) of workspace for the N-D problem over axes[0..dims),
// batch B, nin inputs (2: f and g).
static int64_t ws_elems(int dims, const Axis* ax, int64_t B, int nin = 2)
{
    if (dims == 1) {
        const Axis& a = ax[0];
        int64_t m1 = 0, m2 = 0;
        route(a, B, a.dtype, &m1, &m2);
        if (m1 == 0) return a.D * B * a.m;
        return nin * a.D * B * a.m;
    }
    int64_t Cn = 1, Cf = 1, Cw = 1;
    for (int i = 1; i < dims; ++i) { Cn *= ax[i].L; Cf *= ax[i].Lf; Cw *= ax[i].Lw; }
    const Axis& a = ax[0];
    const int64_t rows = a.D * B * a.m;
    return rows * (Cf + (nin - 1) * Cn + Cw) + ws_elems(dims - 1, ax + 1, rows, nin);
}

static size_t ws_bytes(int dims, const Axis* ax, int64_t B, size_t esz, int ncopy, int nin = 2)
{
    int64_t tot = 1;
    for (int i = 0; i < dims; ++i) tot *= ax[i].L;
    size_t b = 0;
    b += (size_t)ncopy * align_up((size_t)(B * tot) * esz);
    b += align_up((size_t)ws_elems(dims, ax, B, nin) * esz);
    return b + 256;
}

// ------------------------------------------------------------- drivers

#define HDC_TRY(x)                                  \
    do {                                            \
        cudaError_t _e = (x);                       \
        if (_e != cudaSuccess) return _e;           \
    } while (0)

// The inputs of one convolution: n = 2 is f (x[0]) and g (x[1]), possibly
// of unequal lengths; n > 2 is a multi-convolution of equal-length inputs,
// op 0 the n-fold product, op 1 the sum of pairwise products.
template <typename T> struct Ins {
    const cx<T>* x[kMaxInputs];
    int n;
    int op;
};

// Whole convolutions on thread-block clusters (launch_conv_cluster) for a
// few short rows (B rows of C blocks each at most the SM count), where they
// are the faster route.  Measured on single rows with L2 evicted before each
// call: a cluster residue costs about 11 us in FP64 (twice that above 4096
// points), the launch about 17 us; a pass of the split route's four kernels
// about 50 us whatever its size.  So (mode 1) in FP64 the cluster takes
// residues of 256 .. 8192 points when q u <= 2 passes + 1 (u = 1 up to 4096
// points, else 2; passes = ceil(q / D)): explicit padding up to 8192
// points, q = 2 in one pass up to 4096, and every residue count when D = 1
// runs the split route's passes one after another (the L = 1024 configuration
// with (512, 2, 4, 1): 70 against 189 us).  FP32, four times cheaper per
// split-route pass, takes it for one residue up to 16384 points and for D = 1
// multi-pass calls.  Residues of at most 4096 points (powers of two) run
// their transforms as warp shuffles (FP64: 21 us for L = 1024 with
// m = 2048, 48 us on the split route; FP32: 17 us with m = 1024, q = 2,
// against 31 us), and take the cluster in either precision up to q = 4.
template <typename T> static bool use_cluster(const Axis& a, int64_t B)
{
    const int mode = cluster_route_mode();
    if (mode == 0 || a.m < 256) return false;
    int C = 0;
    int64_t m1 = 0, m2 = 0;
    bool warp = false;
    if (!cluster_shape<T>(a.m, a.pout, a.q, a.p, &C, &m1, &m2, nullptr, &warp)) return false;
    if (B * C > (int64_t)sm_count()) return false;
    if (mode == 2) return true;
    const int64_t passes = (a.q + a.D - 1) / a.D;
    if (warp && a.q <= 4) return true;
    if (sizeof(T) == 8) {
        if (a.m > 8192) return false;
        const int64_t u = a.m > 4096 ? 2 : 1;
        return a.q * u <= 2 * passes + 1;
    }
    if (a.m > 16384) return false;
    return a.q == 1 || (passes > 1 && a.q <= 2 * passes + 1);
}

// 1-D convolution of B rows (input row strides ld_f for x[0], ld_g for the
// others, output row stride ldo) along a contiguous axis; outputs
// [a.o, a.o + a.Lw) of every row.  Residues [r_lo, r_hi) of g only (all:
// 0, q): the result is that range's share of the sum over residues, already
// scaled by 1/N, so the shares of disjoint ranges add up to the convolution.
template <typename T>
static cudaError_t run_rows(const Ins<T>& in, cx<T>* out, int64_t B, int64_t ld_f, int64_t ld_g, int64_t ldo,
                            const Axis& a, cx<T>* ws, cudaStream_t st, int64_t r_lo = 0, int64_t r_hi = -1)
{
    const double scale = 1.0 / (double)a.N;
    if (r_hi < 0) r_hi = a.q;
    const cx<T>* f = in.x[0];
    const cx<T>* g = in.x[1];
    if (in.n == 2 && a.lam == 1 && a.Lf == a.L && use_cluster<T>(a, B))
        return launch_conv_cluster<T>(f, g, out, B, ld_f, ld_g, ldo, a.L, a.o, a.o + a.Lw, a.m, a.p, a.q, r_lo, r_hi,
                                      scale, st);
    int64_t m1 = 0, m2 = 0;
    route(a, B, a.dtype, &m1, &m2);
    if (m1 == 0) {
        for (int64_t r0 = r_lo; r0 < r_hi; r0 += a.D) {
            const int64_t Dp = (a.D < r_hi - r0) ? a.D : (r_hi - r0);
            const int first = (r0 == r_lo), last = (r0 + Dp >= r_hi);
            if (in.n > 2)
                HDC_TRY(launch_residue_rows_multi<T>(in.x, in.n, in.op, ws, B, ld_g, a.L, a.m, a.p, a.q, r0, Dp, st));
            else if (a.lam == 1 && a.Lf <= a.L)
                HDC_TRY(launch_residue_rows<T>(f, g, ws, B, ld_f, ld_g, a.Lf, a.L, a.m, a.p, a.q, r0, Dp, st));
            else if (a.lam == 1) // one transform size: the fold runs over the
                                 // longer input's blocks, so (as the inputs
                                 // commute) the longer one goes second
                HDC_TRY(launch_residue_rows<T>(g, f, ws, B, ld_g, ld_f, a.L, a.Lf, a.m, a.pf, a.q, r0, Dp, st));
            else
                HDC_TRY(launch_residue_rows_lam<T>(f, g, ws, B, ld_f, ld_g, a.Lf, a.L, a.mf, a.lam, a.pf, a.p, a.q,
                                                   r0, Dp, st));
            HDC_TRY(launch_unfold<T>(out, ws, B, ldo, 1, a.m, a.pout, a.q, a.N, 1, 0, a.o, a.o + a.Lw, r0,
                                     Dp, first, last, scale, st));
        }
        return cudaSuccess;
    }
    // m = m1 m2: fold + m1-point FFTs along the strided view [p m1][m2] with the
    // inner twiddle zeta_m^{l1 s2}; m2-point row transforms, product and
    // inverse; inverse m1-point FFTs and unfold (one fused pass for one residue
    // per pass when there are enough column tiles).  With lam > 1, f's transform
    // splits as (m1 / lam) m2 and its row l1' of residue q l + r lands on row
    // lam l1' + l, next to the row of g it multiplies.  Input i works in
    // y[i] = ws + i D B m; the product lands in y[0].
    cx<T>* y[kMaxInputs];
    for (int i = 0; i < in.n; ++i) y[i] = ws + (int64_t)i * a.D * B * a.m;
    for (int64_t r0 = r_lo; r0 < r_hi; r0 += a.D) {
        const int64_t Dg = (a.D < r_hi - r0) ? a.D : (r_hi - r0);
        const int first = (r0 == r_lo), last = (r0 + Dg >= r_hi);
        if (in.n > 2) {
            ColSide<T> sides[kMaxInputs];
            for (int i = 0; i < in.n; ++i) sides[i] = ColSide<T>{ in.x[i], y[i], ld_g, a.L, (int)a.p, (int)a.q, 0, 1 };
            HDC_TRY(launch_fold_fft_cols<T>(sides, in.n, B, m2, m1, a.N, m2, 1, r0, Dg, 1, st));
            HDC_TRY(launch_residue_rows_multi<T>(y, in.n, in.op, y[0], Dg * B * m1, m2, m2, m2, 1, 1, 0, 1, st));
        } else {
            const ColSide<T> sf{ f, y[0], ld_f, a.Lf, (int)a.pf, (int)(a.q * a.lam), (int)a.q, (int)a.lam };
            const ColSide<T> sg{ g, y[1], ld_g, a.L, (int)a.p, (int)a.q, 0, 1 };
            if (a.lam == 1) {
                const ColSide<T> both[2] = { sf, sg };
                HDC_TRY(launch_fold_fft_cols<T>(both, 2, B, m2, m1, a.N, m2, 1, r0, Dg, 1, st));
            } else {
                HDC_TRY(launch_fold_fft_cols<T>(&sg, 1, B, m2, m1, a.N, m2, 1, r0, Dg, 1, st));
                HDC_TRY(launch_fold_fft_cols<T>(&sf, 1, B, m2, m1 / a.lam, a.N, m2, 1, r0, Dg, 1, st));
            }
            HDC_TRY(launch_residue_rows<T>(y[0], y[1], y[0], Dg * B * m1, m2, m2, m2, m2, m2, 1, 1, 0, 1, st));
        }
        HDC_TRY(launch_ifft_unfold<T>(y[0], out, B, ldo, m2, m1, a.pout, a.q, a.N, m2, 1, a.o, a.o + a.Lw, r0, Dg,
                                      first, last, scale, 1, st));
    }
    return cudaSuccess;
}

// N-D: residues of axis 0 (strided; Cn, Cf = products of the inner extents
// of g and f, Cw of the inner output extents), the inner (N-1)-D
// convolution on every transformed row, inverse and unfold of the window of
// axis 0.  f's rows are placed next to the rows of g they multiply (residue
// matching along axis 0 when lam > 1).
template <typename T>
static cudaError_t run_nd(int dims, const Ins<T>& in, cx<T>* out, int64_t B, const Axis* ax, cx<T>* ws,
                          cudaStream_t st, int64_t r_lo = 0, int64_t r_hi = -1)
{
    if (dims == 1) return run_rows<T>(in, out, B, ax[0].Lf, ax[0].L, ax[0].Lw, ax[0], ws, st, r_lo, r_hi);
    if (r_hi < 0) r_hi = ax[0].q;
    int64_t Cn = 1, Cf = 1, Cw = 1;
    for (int i = 1; i < dims; ++i) { Cn *= ax[i].L; Cf *= ax[i].Lf; Cw *= ax[i].Lw; }
    const Axis& a = ax[0];
    const int64_t rows = a.D * B * a.m;
    Ins<T> w;
    w.n = in.n;
    w.op = in.op;
    cx<T>* wi[kMaxInputs];
    wi[0] = ws;
    for (int i = 1; i < in.n; ++i) wi[i] = ws + rows * Cf + (int64_t)(i - 1) * rows * Cn;
    for (int i = 0; i < in.n; ++i) w.x[i] = wi[i];
    cx<T>* wh = ws + rows * Cf + (int64_t)(in.n - 1) * rows * Cn;
    cx<T>* inner = wh + rows * Cw;
    const int64_t ostride = a.Lw * Cw;
    const double scale = 1.0 / (double)a.N;
    for (int64_t r0 = r_lo; r0 < r_hi; r0 += a.D) {
        const int64_t Dg = (a.D < r_hi - r0) ? a.D : (r_hi - r0);
        const int first = (r0 == r_lo), last = (r0 + Dg >= r_hi);
        ColSide<T> sides[kMaxInputs];
        sides[0] = ColSide<T>{ in.x[0], wi[0], a.Lf * Cf, a.Lf * Cf, (int)a.pf, (int)(a.q * a.lam), (int)a.q,
                               (int)a.lam };
        for (int i = 1; i < in.n; ++i) sides[i] = ColSide<T>{ in.x[i], wi[i], a.L * Cn, a.L * Cn, (int)a.p, (int)a.q, 0, 1 };
        if (a.lam == 1 && Cf == Cn) {
            HDC_TRY(launch_fold_fft_cols<T>(sides, in.n, B, Cn, a.m, a.N, 1, 0, r0, Dg, 0, st));
        } else {
            HDC_TRY(launch_fold_fft_cols<T>(&sides[1], 1, B, Cn, a.m, a.N, 1, 0, r0, Dg, 0, st));
            HDC_TRY(launch_fold_fft_cols<T>(&sides[0], 1, B, Cf, a.mf, a.N, 1, 0, r0, Dg, 0, st));
        }
        HDC_TRY(run_nd<T>(dims - 1, w, wh, Dg * B * a.m, ax + 1, inner, st));
        HDC_TRY(launch_ifft_unfold<T>(wh, out, B, ostride, Cw, a.m, a.pout, a.q, a.N, 1, 0, a.o * Cw,
                                      (a.o + a.Lw) * Cw, r0, Dg, first, last, scale, 0, st));
    }
    return cudaSuccess;
}

// ------------------------------------------------------- real inputs
// f and g real, packed as z = f + i g; only the residues r <= q / 2 of the
// first axis are formed (r' = q - r is the conjugate partner), so D counts
// kept residues per pass.

static int64_t kept_residues(const Axis& a) { return a.q / 2 + 1; }

static int64_t ws_elems_real(int dims, const Axis* ax, int64_t B)
{
    const Axis& a = ax[0];
    const int64_t D = a.D < kept_residues(a) ? a.D : kept_residues(a);
    if (dims == 1) {
        int64_t m1 = 0, m2 = 0;
        route(a, B, a.dtype, &m1, &m2);
        return (m1 == 0 ? 1 : 3) * D * B * a.m;
    }
    int64_t Cn = 1, Cw = 1;
    for (int i = 1; i < dims; ++i) { Cn *= ax[i].L; Cw *= ax[i].Lw; }
    const int64_t rows = D * B * a.m;
    return rows * (4 * Cn + Cw) + ws_elems(dims - 1, ax + 1, rows);
}

static size_t ws_bytes_real(int dims, const Axis* ax, int64_t B, size_t esz)
{
    int64_t tot = 1;
    for (int i = 0; i < dims; ++i) tot *= ax[i].L;
    return align_up((size_t)(B * tot) * esz) + align_up((size_t)ws_elems_real(dims, ax, B) * esz) + 256;
}

template <typename T>
static cudaError_t run_rows_real(const cx<T>* z, T* out, int64_t B, const Axis& a, cx<T>* ws, cudaStream_t st)
{
    const double scale = 1.0 / (double)a.N;
    const int64_t S = kept_residues(a);
    const int64_t D = a.D < S ? a.D : S;
    int64_t m1 = 0, m2 = 0;
    route(a, B, a.dtype, &m1, &m2);
    cx<T>* ya = ws;
    cx<T>* yb = ws + D * B * a.m;
    cx<T>* yh = ws + 2 * D * B * a.m;
    for (int64_t r0 = 0; r0 < S; r0 += D) {
        const int64_t Dp = (D < S - r0) ? D : (S - r0);
        const int first = (r0 == 0), last = (r0 + Dp >= S);
        if (m1 == 0) {
            HDC_TRY(launch_residue_rows_real<T>(z, ya, B, a.L, a.L, a.m, a.p, a.q, r0, Dp, st));
            HDC_TRY(launch_unfold_real<T>(out, ya, B, a.L, 1, a.m, a.pout, a.q, a.N, 1, 0, 0, a.L, r0, Dp, first,
                                          last, scale, st));
            continue;
        }
        ColSide<T> sides[2];
        sides[0] = ColSide<T>{ z, ya, a.L, a.L, (int)a.p, (int)a.q, 0, 1 };
        sides[1] = ColSide<T>{ z, yb, a.L, a.L, (int)a.p, (int)a.q, 0, 1 };
        sides[1].rneg = 1;
        HDC_TRY(launch_fold_fft_cols<T>(sides, 2, B, m2, m1, a.N, m2, 1, r0, Dp, 1, st));
        HDC_TRY(launch_rows_real_pair<T>(ya, yb, yh, B, m1, m2, a.q, r0, Dp, st));
        HDC_TRY(launch_ifft_cols<T>(yh, B, m2, m1, a.q, a.N, Dp, 1, st));
        HDC_TRY(launch_unfold_real<T>(out, yh, B, a.L, m2, m1, a.pout, a.q, a.N, m2, 1, 0, a.L, r0, Dp, first, last,
                                      scale, st));
    }
    return cudaSuccess;
}

template <typename T>
static cudaError_t run_nd_real(int dims, const cx<T>* z, T* out, int64_t B, const Axis* ax, cx<T>* ws,
                               cudaStream_t st)
{
    if (dims == 1) return run_rows_real<T>(z, out, B, ax[0], ws, st);
    const Axis& a = ax[0];
    int64_t Cn = 1, Cw = 1;
    for (int i = 1; i < dims; ++i) { Cn *= ax[i].L; Cw *= ax[i].Lw; }
    const int64_t S = kept_residues(a);
    const int64_t D = a.D < S ? a.D : S;
    const int64_t rows = D * B * a.m;
    cx<T>* wa = ws;
    cx<T>* wb = wa + rows * Cn;
    cx<T>* wf = wb + rows * Cn;
    cx<T>* wg = wf + rows * Cn;
    cx<T>* wh = wg + rows * Cn;
    cx<T>* inner = wh + rows * Cw;
    const double scale = 1.0 / (double)a.N;
    Ins<T> in;
    in.n = 2;
    in.op = 0;
    in.x[0] = wf;
    in.x[1] = wg;
    for (int64_t r0 = 0; r0 < S; r0 += D) {
        const int64_t Dp = (D < S - r0) ? D : (S - r0);
        const int first = (r0 == 0), last = (r0 + Dp >= S);
        ColSide<T> sides[2];
        sides[0] = ColSide<T>{ z, wa, a.L * Cn, a.L * Cn, (int)a.p, (int)a.q, 0, 1 };
        sides[1] = ColSide<T>{ z, wb, a.L * Cn, a.L * Cn, (int)a.p, (int)a.q, 0, 1 };
        sides[1].rneg = 1;
        HDC_TRY(launch_fold_fft_cols<T>(sides, 2, B, Cn, a.m, a.N, 1, 0, r0, Dp, 0, st));
        HDC_TRY(launch_pair_rows_real<T>(wa, wb, wf, wg, B, Cn, a.m, a.q, r0, Dp, st));
        HDC_TRY(run_nd<T>(dims - 1, in, wh, Dp * B * a.m, ax + 1, inner, st));
        HDC_TRY(launch_ifft_cols<T>(wh, B, Cw, a.m, a.q, a.N, Dp, 0, st));
        HDC_TRY(launch_unfold_real<T>(out, wh, B, a.L * Cw, Cw, a.m, a.pout, a.q, a.N, 1, 0, 0, a.L * Cw, r0, Dp,
                                      first, last, scale, st));
    }
    return cudaSuccess;
}

template <typename T>
static int conv_nd_real(int dims, const void* f, const void* g, void* h, const Axis* ax, int64_t B, void* ws,
                        size_t ws_bytes_given, cudaStream_t st)
{
    using V = cx<T>;
    const size_t need = ws_bytes_real(dims, ax, B, sizeof(V));
    if (!preparing() && (ws == nullptr || ws_bytes_given < need)) return HDC_ERR_WORKSPACE;
    int64_t tot = B;
    for (int i = 0; i < dims; ++i) tot *= ax[i].L;
    uintptr_t base = ((uintptr_t)ws + 255) & ~(uintptr_t)255;
    V* z = (V*)base;
    V* w = (V*)(base + align_up((size_t)tot * sizeof(V)));
    if (!preparing() && launch_pack_real<T>((const T*)f, (const T*)g, z, tot, st) != cudaSuccess) return HDC_ERR_CUDA;
    cudaError_t e = run_nd_real<T>(dims, z, (T*)h, B, ax, w, st);
    return cuda_rc(e);
}

template <typename T>
static int conv_nd(int dims, const void* f, const void* g, void* h, const Axis* ax, int inplace,
                   int64_t B, void* ws, size_t ws_bytes_given, cudaStream_t st, int64_t r_lo = 0,
                   int64_t r_hi = -1)
{
    using V = cx<T>;
    int64_t tot = 1;
    bool same_shape = true;
    for (int i = 0; i < dims; ++i) {
        tot *= ax[i].L;
        same_shape = same_shape && ax[i].o == 0 && ax[i].Lw == ax[i].L && ax[i].Lf == ax[i].L && ax[i].lam == 1;
    }
    const bool af = (h == f), ag = (h == g);
    if ((af || ag) && (!inplace || !same_shape)) return HDC_ERR_PARAM;
    const int ncopy = (int)af + (int)(ag && g != f);
    const size_t need = ws_bytes(dims, ax, B, sizeof(V), ncopy);
    if (!preparing() && (ws == nullptr || ws_bytes_given < need)) return HDC_ERR_WORKSPACE;
    uintptr_t base = ((uintptr_t)ws + 255) & ~(uintptr_t)255;
    const V* fin = (const V*)f;
    const V* gin = (const V*)g;
    const size_t arr = (size_t)(B * tot) * sizeof(V);
    if (af && !preparing()) {
        if (cudaMemcpyAsync((void*)base, f, arr, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return HDC_ERR_CUDA;
        fin = (const V*)base;
        if (g == f) gin = fin;
        base += align_up(arr);
    }
    if (ag && g != f && !preparing()) {
        if (cudaMemcpyAsync((void*)base, g, arr, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return HDC_ERR_CUDA;
        gin = (const V*)base;
        base += align_up(arr);
    }
    Ins<T> in;
    in.n = 2;
    in.op = 0;
    in.x[0] = fin;
    in.x[1] = gin;
    cudaError_t e = run_nd<T>(dims, in, (V*)h, B, ax, (V*)base, st, r_lo, r_hi);
    return cuda_rc(e);
}

// Multi-convolution of n equal-shape inputs (device pointers, distinct from
// h), operator op; workspace of ws_bytes(..., nin = n).
template <typename T>
static int conv_nd_multi(int dims, int n, int op, const void* const* xs, void* h, const Axis* ax, int64_t B,
                         void* ws, size_t ws_bytes_given, cudaStream_t st)
{
    using V = cx<T>;
    const size_t need = ws_bytes(dims, ax, B, sizeof(V), 0, n);
    if (!preparing() && (ws == nullptr || ws_bytes_given < need)) return HDC_ERR_WORKSPACE;
    uintptr_t base = ((uintptr_t)ws + 255) & ~(uintptr_t)255;
    Ins<T> in;
    in.n = n;
    in.op = op;
    for (int i = 0; i < n; ++i) in.x[i] = (const V*)xs[i];
    cudaError_t e = run_nd<T>(dims, in, (V*)h, B, ax, (V*)base, st);
    return cuda_rc(e);
}

static int resolve_all(int dims, const int64_t* L, const int64_t* M, const int64_t* m, const int64_t* p,
                       const int64_t* q, const int64_t* D, int dtype, Axis* ax, const int64_t* o = nullptr,
                       const int64_t* Lw = nullptr)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !L || !M || !m) return HDC_ERR_PARAM;
    for (int i = 0; i < dims; ++i) {
        int rc = resolve_axis(L[i], M[i], m[i], p ? p[i] : 0, q ? q[i] : 0, D ? D[i] : 0, dtype, &ax[i],
                              o ? o[i] : 0, Lw ? Lw[i] : -1);
        if (rc != HDC_OK) return rc;
        // an axis with inner axes runs its whole m-point FFT in one column tile
        if (i < dims - 1 && m[i] > (dtype == HDC_C128 ? max_col_fft<double>() : max_col_fft<float>()))
            return HDC_ERR_UNSUPPORTED_SIZE;
    }
    return HDC_OK;
}

static int resolve_all_uneq(int dims, const int64_t* Lf, const int64_t* Lg, const int64_t* M, const int64_t* m,
                            const int64_t* lam, const int64_t* D, const int64_t* o, const int64_t* Lw, int dtype,
                            Axis* ax)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !Lf || !Lg || !m) return HDC_ERR_PARAM;
    for (int i = 0; i < dims; ++i) {
        int rc = resolve_axis_uneq(Lf[i], Lg[i], M ? M[i] : 0, m[i], lam ? lam[i] : 1, D ? D[i] : 0, dtype, &ax[i],
                                   o ? o[i] : 0, Lw ? Lw[i] : -1);
        if (rc != HDC_OK) return rc;
        if (i < dims - 1 && ax[i].m > (dtype == HDC_C128 ? max_col_fft<double>() : max_col_fft<float>()))
            return HDC_ERR_UNSUPPORTED_SIZE;
    }
    return HDC_OK;
}

// Multi-convolution of n equal-length inputs: the first L outputs of the
// n-fold convolution per axis are alias-free when M >= n (L - 1) + 1; the
// sum of pairwise products (n even) needs the two-input M >= 2 L - 1.
static int resolve_all_multi(int dims, int n, int op, const int64_t* L, const int64_t* M, const int64_t* m,
                             const int64_t* p, const int64_t* q, const int64_t* D, int dtype, Axis* ax)
{
    if (n < 2 || n > kMaxInputs || dims < 1 || dims > HDC_MAX_DIMS || !L || !m) return HDC_ERR_PARAM;
    if (op != HDC_MULTI_PRODUCT && op != HDC_MULTI_DOT) return HDC_ERR_PARAM;
    if (op == HDC_MULTI_DOT && (n & 1)) return HDC_ERR_PARAM;
    const int fold = op == HDC_MULTI_PRODUCT ? n : 2;
    int64_t Mv[HDC_MAX_DIMS];
    for (int i = 0; i < dims; ++i) {
        if (L[i] < 1) return HDC_ERR_PARAM;
        Mv[i] = (M && M[i] > 0) ? M[i] : fold * (L[i] - 1) + 1;
        if (Mv[i] < fold * (L[i] - 1) + 1) return HDC_ERR_ALIAS;
    }
    return resolve_all(dims, L, Mv, m, p, q, D, dtype, ax);
}

} // namespace hdc

using namespace hdc;

// ------------------------------------------------------------------ ABI

HDC_EXPORT int hdc_last_cuda_error(void) { return g_last_cuda_error.load(); }

HDC_EXPORT const char* hdc_last_cuda_error_name(void)
{
    return cudaGetErrorName((cudaError_t)g_last_cuda_error.load());
}

HDC_EXPORT const char* hdc_strerror(int status)
{
    switch (status) {
    case HDC_OK: return "ok";
    case HDC_ERR_PARAM: return "invalid or inconsistent parameters";
    case HDC_ERR_ALIAS: return "padding too small: M < 2L-1 would alias";
    case HDC_ERR_UNSUPPORTED_SIZE: return "unsupported size (m must be 2^a 3^b 5^c 7^d within the limits)";
    case HDC_ERR_DTYPE: return "unknown dtype";
    case HDC_ERR_ALLOC: return "device allocation failed";
    case HDC_ERR_CUDA: return "CUDA runtime error";
    case HDC_ERR_TIMEOUT: return "device wait timed out";
    case HDC_ERR_NOT_TUNED: return "no tuning record or predictor for this request";
    case HDC_ERR_WORKSPACE: return "workspace missing or too small";
    case HDC_ERR_NOT_PREPARED: return "twiddle tables not made for this problem: call hdc_prepare* or create a plan first";
    default: return "unknown status";
    }
}

HDC_EXPORT int hdc_version(void) { return 100; }

HDC_EXPORT int hdc_is_good_size(int64_t n) { return good_size(n) ? 1 : 0; }

HDC_EXPORT int64_t hdc_next_good_size(int64_t n)
{
    if (n < 1) return -1;
    for (int64_t k = n; k < ((int64_t)1 << 62); ++k)
        if (good_size(k)) return k;
    return -1;
}

HDC_EXPORT int hdc_derive_params(int64_t L, int64_t M, int64_t m, int64_t* p, int64_t* q)
{
    if (L < 1 || M < 1 || m < 1 || !p || !q) return HDC_ERR_PARAM;
    *p = ceil_div(L, m);
    *q = ceil_div(M, m);
    return HDC_OK;
}

HDC_EXPORT int hdc_explicit_params(int64_t L, int64_t M, int64_t* m, int64_t* p, int64_t* q)
{
    if (L < 1 || M < 1 || !m || !p || !q) return HDC_ERR_PARAM;
    *m = hdc_next_good_size(M);
    if (*m < 0) return HDC_ERR_UNSUPPORTED_SIZE;
    *p = 1;
    *q = 1;
    return HDC_OK;
}

HDC_EXPORT int hdc_validate_axis(int64_t L, int64_t M, int64_t m, int64_t p, int64_t q, int64_t D, int dtype,
                                 int64_t* p_out, int64_t* q_out, int64_t* D_out)
{
    Axis a;
    int rc = resolve_axis(L, M, m, p, q, D, dtype, &a);
    if (rc != HDC_OK) return rc;
    if (p_out) *p_out = a.p;
    if (q_out) *q_out = a.q;
    if (D_out) *D_out = a.D;
    return HDC_OK;
}

HDC_EXPORT int64_t hdc_max_fft_size(int dtype) { return max_fft(dtype); }
HDC_EXPORT int64_t hdc_max_outer_fft_size(int dtype)
{
    return dtype == HDC_C128 ? max_col_fft<double>() : max_col_fft<float>();
}
HDC_EXPORT int64_t hdc_max_padded_size(int dtype) { return max_padded(dtype); }

template <typename T> static int fft_stages(int64_t n, int kind, int* radices, int cap)
{
    const int64_t lim = kind == HDC_FFT_COLS ? max_col_fft<T>() : max_row_fft<T>();
    if (n > lim) return HDC_ERR_UNSUPPORTED_SIZE;
    const bool r16ok = kind == HDC_FFT_COLS || (kind == HDC_FFT_ROWS && rows_r16(n));
    const FftPlan fp = fft_plan<T>(n, r16ok);
    if (fp.nst > cap) return HDC_ERR_PARAM;
    for (int s = 0; s < fp.nst; ++s) radices[s] = fp.rad[s];
    return fp.nst;
}

HDC_EXPORT int hdc_fft_stages(int64_t n, int dtype, int kind, int* radices, int cap)
{
    if (!radices || cap < 0 || kind < HDC_FFT_ROWS || kind > HDC_FFT_OTHER) return HDC_ERR_PARAM;
    if (dtype != HDC_C128 && dtype != HDC_C64) return HDC_ERR_DTYPE;
    if (n < 1 || !hdc_is_good_size(n)) return HDC_ERR_UNSUPPORTED_SIZE;
    return dtype == HDC_C128 ? fft_stages<double>(n, kind, radices, cap) : fft_stages<float>(n, kind, radices, cap);
}

HDC_EXPORT int hdc_workspace_size(int dims, const int64_t* L, const int64_t* M, const int64_t* m,
                                  const int64_t* p, const int64_t* q, const int64_t* D, int dtype,
                                  int64_t batch, int inplace, size_t* bytes)
{
    if (!bytes || batch < 0) return HDC_ERR_PARAM;
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    const size_t esz = dtype == HDC_C128 ? 16 : 8;
    *bytes = ws_bytes(dims, ax, batch, esz, inplace ? 2 : 0);
    return HDC_OK;
}

HDC_EXPORT int hdc_convnd(int dims, const void* f, const void* g, void* h, const int64_t* L, const int64_t* M,
                          const int64_t* m, const int64_t* p, const int64_t* q, const int64_t* D, int inplace,
                          int dtype, int64_t batch, void* workspace, size_t ws_bytes_given, void* stream)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    if (!f || !g || !h) return HDC_ERR_PARAM;
    const uintptr_t al = dtype == HDC_C128 ? 15 : 7;
    if (((uintptr_t)f & al) || ((uintptr_t)g & al) || ((uintptr_t)h & al)) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == HDC_C128) return conv_nd<double>(dims, f, g, h, ax, inplace, batch, workspace, ws_bytes_given, st);
    return conv_nd<float>(dims, f, g, h, ax, inplace, batch, workspace, ws_bytes_given, st);
}

HDC_EXPORT int hdc_conv1d(const void* f, const void* g, void* h, int64_t L, int64_t M, int64_t m, int64_t p,
                          int64_t q, int64_t D, int inplace, int dtype, int64_t batch, void* workspace,
                          size_t ws_bytes_given, void* stream)
{
    return hdc_convnd(1, f, g, h, &L, &M, &m, &p, &q, &D, inplace, dtype, batch, workspace, ws_bytes_given,
                      stream);
}

HDC_EXPORT int hdc_conv2d(const void* f, const void* g, void* h, const int64_t L[2], const int64_t M[2],
                          const int64_t m[2], const int64_t p[2], const int64_t q[2], const int64_t D[2],
                          int inplace, int dtype, int64_t batch, void* workspace, size_t ws_bytes_given,
                          void* stream)
{
    return hdc_convnd(2, f, g, h, L, M, m, p, q, D, inplace, dtype, batch, workspace, ws_bytes_given, stream);
}

HDC_EXPORT int hdc_conv3d(const void* f, const void* g, void* h, const int64_t L[3], const int64_t M[3],
                          const int64_t m[3], const int64_t p[3], const int64_t q[3], const int64_t D[3],
                          int inplace, int dtype, int64_t batch, void* workspace, size_t ws_bytes_given,
                          void* stream)
{
    return hdc_convnd(3, f, g, h, L, M, m, p, q, D, inplace, dtype, batch, workspace, ws_bytes_given, stream);
}

HDC_EXPORT int hdc_workspace_size_host(int dims, const int64_t* L, const int64_t* M, const int64_t* m,
                                       const int64_t* p, const int64_t* q, const int64_t* D, int dtype,
                                       int64_t batch, size_t* bytes)
{
    if (!bytes || batch < 0) return HDC_ERR_PARAM;
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    const size_t esz = dtype == HDC_C128 ? 16 : 8;
    int64_t tot = batch;
    for (int i = 0; i < dims; ++i) tot *= ax[i].L;
    *bytes = 3 * align_up((size_t)tot * esz) + ws_bytes(dims, ax, batch, esz, 0) + 256;
    return HDC_OK;
}

HDC_EXPORT int hdc_convnd_host(int dims, const void* f_host, const void* g_host, void* h_host, const int64_t* L,
                               const int64_t* M, const int64_t* m, const int64_t* p, const int64_t* q,
                               const int64_t* D, int dtype, int64_t batch, void* dev_ws, size_t ws_bytes_given,
                               void* stream)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    if (!f_host || !g_host || !h_host) return HDC_ERR_PARAM;
    size_t need = 0;
    rc = hdc_workspace_size_host(dims, L, M, m, p, q, D, dtype, batch, &need);
    if (rc != HDC_OK) return rc;
    if (!dev_ws || ws_bytes_given < need) return HDC_ERR_WORKSPACE;
    const size_t esz = dtype == HDC_C128 ? 16 : 8;
    int64_t tot = batch;
    for (int i = 0; i < dims; ++i) tot *= ax[i].L;
    const size_t arr = (size_t)tot * esz;
    uintptr_t base = ((uintptr_t)dev_ws + 255) & ~(uintptr_t)255;
    void* df = (void*)base;
    void* dg = (void*)(base + align_up(arr));
    void* dh = (void*)(base + 2 * align_up(arr));
    void* w = (void*)(base + 3 * align_up(arr));
    const size_t wbytes = ws_bytes_given - (size_t)((uintptr_t)w - (uintptr_t)dev_ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(df, f_host, arr, cudaMemcpyHostToDevice, st) != cudaSuccess) return HDC_ERR_CUDA;
    if (cudaMemcpyAsync(dg, g_host, arr, cudaMemcpyHostToDevice, st) != cudaSuccess) return HDC_ERR_CUDA;
    rc = dtype == HDC_C128 ? conv_nd<double>(dims, df, dg, dh, ax, 0, batch, w, wbytes, st)
                           : conv_nd<float>(dims, df, dg, dh, ax, 0, batch, w, wbytes, st);
    if (rc != HDC_OK) return rc;
    if (cudaMemcpyAsync(h_host, dh, arr, cudaMemcpyDeviceToHost, st) != cudaSuccess) return HDC_ERR_CUDA;
    return HDC_OK;
}

HDC_EXPORT int hdc_workspace_size_window(int dims, const int64_t* L, const int64_t* M, const int64_t* m,
                                         const int64_t* p, const int64_t* q, const int64_t* D, const int64_t* o,
                                         const int64_t* Lw, int dtype, int64_t batch, size_t* bytes)
{
    if (!bytes || batch < 0 || !o || !Lw) return HDC_ERR_PARAM;
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax, o, Lw);
    if (rc != HDC_OK) return rc;
    *bytes = ws_bytes(dims, ax, batch, dtype == HDC_C128 ? 16 : 8, 0);
    return HDC_OK;
}

HDC_EXPORT int hdc_convnd_window(int dims, const void* f, const void* g, void* h, const int64_t* L, const int64_t* M,
                                 const int64_t* m, const int64_t* p, const int64_t* q, const int64_t* D,
                                 const int64_t* o, const int64_t* Lw, int dtype, int64_t batch, void* workspace,
                                 size_t ws_bytes_given, void* stream)
{
    if (!o || !Lw) return HDC_ERR_PARAM;
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax, o, Lw);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    if (!f || !g || !h) return HDC_ERR_PARAM;
    const uintptr_t al = dtype == HDC_C128 ? 15 : 7;
    if (((uintptr_t)f & al) || ((uintptr_t)g & al) || ((uintptr_t)h & al)) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == HDC_C128) return conv_nd<double>(dims, f, g, h, ax, 0, batch, workspace, ws_bytes_given, st);
    return conv_nd<float>(dims, f, g, h, ax, 0, batch, workspace, ws_bytes_given, st);
}

// The half-stored route of the centered Hermitian convolution: the outer
// axis (kx, 2K - 1 points shifted by c, padded to M = 3K - 2, window
// [c, 3c]) through the residue kernels of the N-D route on the K stored
// half columns; the inner axis (ky) through launch_hermitian_rows, which
// transforms the two fields of a row in one packed transform, multiplies the
// real fields and inverse-transforms a pair of rows at once.
template <typename T> static int herm_resolve(int64_t K, const int64_t* m, const int64_t* D, int dtype, Axis* ax,
                                              Axis* ay)
{
    const int64_t c = K - 1, L = 2 * K - 1, M = 3 * K - 2;
    int rc = resolve_axis(L, M, m[0], 0, 0, D ? D[0] : 0, dtype, ax, c, L);
    if (rc != HDC_OK) return rc;
    rc = resolve_axis(L, M, m[1], 0, 0, 0, dtype, ay, c, L);
    if (rc != HDC_OK) return rc;
    // the outer transform runs in one column tile; the inner one, with both
    // packed rows and the pair's 2K - 1 outputs, in one block's shared memory
    if (m[0] > max_col_fft<T>() || m[1] > max_row_fft<T>()) return HDC_ERR_UNSUPPORTED_SIZE;
    if ((2 * smem_len<cx<T>>(2 * m[1]) + 2 * K - 1) * (int64_t)sizeof(cx<T>) > 200 * 1024)
        return HDC_ERR_UNSUPPORTED_SIZE;
    return HDC_OK;
}

static int herm_resolve_any(int64_t K, const int64_t* m, const int64_t* D, int dtype, Axis* ax, Axis* ay)
{
    if (K < 1 || !m) return HDC_ERR_PARAM;
    if (dtype == HDC_C128) return herm_resolve<double>(K, m, D, dtype, ax, ay);
    if (dtype == HDC_C64) return herm_resolve<float>(K, m, D, dtype, ax, ay);
    return HDC_ERR_DTYPE;
}

static size_t herm_ws_bytes(const Axis& ax, int64_t K, int64_t B, size_t esz)
{
    return align_up((size_t)(3 * ax.D * B * ax.m * K) * esz) + 256;
}

template <typename T>
static cudaError_t run_hermitian(const cx<T>* f, const cx<T>* g, cx<T>* out, int64_t B, int64_t K, const Axis& ax,
                                 const Axis& ay, cx<T>* ws, cudaStream_t st)
{
    const int64_t Cn = K, L = 2 * K - 1;
    const int64_t rows = ax.D * B * ax.m;
    cx<T>* wf = ws;
    cx<T>* wg = wf + rows * Cn;
    cx<T>* wh = wg + rows * Cn;
    const double scale = 1.0 / (double)ax.N;
    for (int64_t r0 = 0; r0 < ax.q; r0 += ax.D) {
        const int64_t Dg = (ax.D < ax.q - r0) ? ax.D : (ax.q - r0);
        const int first = (r0 == 0), last = (r0 + Dg >= ax.q);
        const ColSide<T> sides[2] = { ColSide<T>{ f, wf, L * Cn, L * Cn, (int)ax.p, (int)ax.q, 0, 1 },
                                      ColSide<T>{ g, wg, L * Cn, L * Cn, (int)ax.p, (int)ax.q, 0, 1 } };
        HDC_TRY(launch_fold_fft_cols<T>(sides, 2, B, Cn, ax.m, ax.N, 1, 0, r0, Dg, 0, st));
        HDC_TRY(launch_hermitian_rows<T>(wf, wg, wh, Dg * B, B, ax.m, K, ay.m, ay.q, ax.N, ax.q, r0, st));
        HDC_TRY(launch_ifft_unfold<T>(wh, out, B, L * Cn, Cn, ax.m, ax.pout, ax.q, ax.N, 1, 0, ax.o * Cn,
                                      (ax.o + ax.Lw) * Cn, r0, Dg, first, last, scale, 0, st));
    }
    return cudaSuccess;
}

HDC_EXPORT int hdc_workspace_size_hermitian(int64_t K, const int64_t* m, const int64_t* D, int dtype, int64_t batch,
                                            size_t* bytes)
{
    if (!bytes || batch < 0) return HDC_ERR_PARAM;
    Axis ax, ay;
    int rc = herm_resolve_any(K, m, D, dtype, &ax, &ay);
    if (rc != HDC_OK) return rc;
    *bytes = herm_ws_bytes(ax, K, batch, dtype == HDC_C128 ? 16 : 8);
    return HDC_OK;
}

HDC_EXPORT int hdc_conv2d_hermitian(const void* f, const void* g, void* h, int64_t K, const int64_t* m,
                                    const int64_t* D, int dtype, int64_t batch, void* workspace,
                                    size_t ws_bytes_given, void* stream)
{
    Axis ax, ay;
    int rc = herm_resolve_any(K, m, D, dtype, &ax, &ay);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    if (!preparing()) {
        if (!f || !g || !h || h == f || h == g) return HDC_ERR_PARAM;
        const uintptr_t al = dtype == HDC_C128 ? 15 : 7;
        if (((uintptr_t)f & al) || ((uintptr_t)g & al) || ((uintptr_t)h & al)) return HDC_ERR_PARAM;
        if (!workspace || ws_bytes_given < herm_ws_bytes(ax, K, batch, dtype == HDC_C128 ? 16 : 8))
            return HDC_ERR_WORKSPACE;
    }
    uintptr_t base = ((uintptr_t)workspace + 255) & ~(uintptr_t)255;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = dtype == HDC_C128
                        ? run_hermitian<double>((const cx<double>*)f, (const cx<double>*)g, (cx<double>*)h, batch, K,
                                                ax, ay, (cx<double>*)base, st)
                        : run_hermitian<float>((const cx<float>*)f, (const cx<float>*)g, (cx<float>*)h, batch, K, ax,
                                               ay, (cx<float>*)base, st);
    return cuda_rc(e);
}

HDC_EXPORT int hdc_convnd_residues(int dims, const void* f, const void* g, void* h, const int64_t* L,
                                   const int64_t* M, const int64_t* m, const int64_t* p, const int64_t* q,
                                   const int64_t* D, int64_t r_lo, int64_t r_hi, int dtype, int64_t batch,
                                   void* workspace, size_t ws_bytes_given, void* stream)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0 || r_lo < 0 || r_hi > ax[0].q || r_lo >= r_hi) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    if (!f || !g || !h || h == f || h == g) return HDC_ERR_PARAM;
    const uintptr_t al = dtype == HDC_C128 ? 15 : 7;
    if (((uintptr_t)f & al) || ((uintptr_t)g & al) || ((uintptr_t)h & al)) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == HDC_C128)
        return conv_nd<double>(dims, f, g, h, ax, 0, batch, workspace, ws_bytes_given, st, r_lo, r_hi);
    return conv_nd<float>(dims, f, g, h, ax, 0, batch, workspace, ws_bytes_given, st, r_lo, r_hi);
}

HDC_EXPORT int hdc_validate_unequal_axis(int64_t Lf, int64_t Lg, int64_t M, int64_t m, int64_t lam, int64_t D,
                                         int dtype, int64_t* pf, int64_t* pg, int64_t* qg, int64_t* D_out)
{
    Axis a;
    int rc = resolve_axis_uneq(Lf, Lg, M, m, lam, D, dtype, &a, 0, -1);
    if (rc != HDC_OK) return rc;
    if (pf) *pf = a.pf;
    if (pg) *pg = a.p;
    if (qg) *qg = a.q;
    if (D_out) *D_out = a.D;
    return HDC_OK;
}

HDC_EXPORT int hdc_workspace_size_unequal(int dims, const int64_t* Lf, const int64_t* Lg, const int64_t* M,
                                          const int64_t* m, const int64_t* lam, const int64_t* D, const int64_t* o,
                                          const int64_t* Lw, int dtype, int64_t batch, size_t* bytes)
{
    if (!bytes || batch < 0) return HDC_ERR_PARAM;
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all_uneq(dims, Lf, Lg, M, m, lam, D, o, Lw, dtype, ax);
    if (rc != HDC_OK) return rc;
    *bytes = ws_bytes(dims, ax, batch, dtype == HDC_C128 ? 16 : 8, 0);
    return HDC_OK;
}

HDC_EXPORT int hdc_convnd_unequal(int dims, const void* f, const void* g, void* h, const int64_t* Lf,
                                  const int64_t* Lg, const int64_t* M, const int64_t* m, const int64_t* lam,
                                  const int64_t* D, const int64_t* o, const int64_t* Lw, int dtype, int64_t batch,
                                  void* workspace, size_t ws_bytes_given, void* stream)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all_uneq(dims, Lf, Lg, M, m, lam, D, o, Lw, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    if (!f || !g || !h || h == f || h == g) return HDC_ERR_PARAM;
    const uintptr_t al = dtype == HDC_C128 ? 15 : 7;
    if (((uintptr_t)f & al) || ((uintptr_t)g & al) || ((uintptr_t)h & al)) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == HDC_C128) return conv_nd<double>(dims, f, g, h, ax, 0, batch, workspace, ws_bytes_given, st);
    return conv_nd<float>(dims, f, g, h, ax, 0, batch, workspace, ws_bytes_given, st);
}

HDC_EXPORT int hdc_workspace_size_multi(int dims, int n, int op, const int64_t* L, const int64_t* M,
                                        const int64_t* m, const int64_t* p, const int64_t* q, const int64_t* D,
                                        int dtype, int64_t batch, size_t* bytes)
{
    if (!bytes || batch < 0) return HDC_ERR_PARAM;
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all_multi(dims, n, op, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    *bytes = ws_bytes(dims, ax, batch, dtype == HDC_C128 ? 16 : 8, 0, n);
    return HDC_OK;
}

HDC_EXPORT int hdc_convnd_multi(int dims, int n, int op, const void* const* inputs, void* h, const int64_t* L,
                                const int64_t* M, const int64_t* m, const int64_t* p, const int64_t* q,
                                const int64_t* D, int dtype, int64_t batch, void* workspace, size_t ws_bytes_given,
                                void* stream)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all_multi(dims, n, op, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0 || !inputs || !h) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    const uintptr_t al = dtype == HDC_C128 ? 15 : 7;
    if ((uintptr_t)h & al) return HDC_ERR_PARAM;
    for (int i = 0; i < n; ++i)
        if (!inputs[i] || inputs[i] == h || ((uintptr_t)inputs[i] & al)) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == HDC_C128)
        return conv_nd_multi<double>(dims, n, op, inputs, h, ax, batch, workspace, ws_bytes_given, st);
    return conv_nd_multi<float>(dims, n, op, inputs, h, ax, batch, workspace, ws_bytes_given, st);
}

HDC_EXPORT int hdc_workspace_size_real(int dims, const int64_t* L, const int64_t* M, const int64_t* m,
                                       const int64_t* p, const int64_t* q, const int64_t* D, int dtype, int64_t batch,
                                       size_t* bytes)
{
    if (!bytes || batch < 0) return HDC_ERR_PARAM;
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    *bytes = ws_bytes_real(dims, ax, batch, dtype == HDC_C128 ? 16 : 8);
    return HDC_OK;
}

HDC_EXPORT int hdc_convnd_real(int dims, const void* f, const void* g, void* h, const int64_t* L, const int64_t* M,
                               const int64_t* m, const int64_t* p, const int64_t* q, const int64_t* D, int dtype,
                               int64_t batch, void* workspace, size_t ws_bytes_given, void* stream)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    if (!f || !g || !h || h == f || h == g) return HDC_ERR_PARAM;
    const uintptr_t al = dtype == HDC_C128 ? 7 : 3;
    if (((uintptr_t)f & al) || ((uintptr_t)g & al) || ((uintptr_t)h & al)) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == HDC_C128) return conv_nd_real<double>(dims, f, g, h, ax, batch, workspace, ws_bytes_given, st);
    return conv_nd_real<float>(dims, f, g, h, ax, batch, workspace, ws_bytes_given, st);
}

// ------------------------------------------------------------ preparation
// Each hdc_prepare* walks the drivers of its convolution call in the
// kTablesPrepare mode: every launcher fetches (and so makes) the tables it
// reads and returns before launching.  The data pointers of that walk are
// distinct stand-in addresses that nothing reads or writes.

static const void* no_data(int k) { return reinterpret_cast<const void*>(((uintptr_t)1 << 40) + ((uintptr_t)k << 20)); }

template <class Run> static int prepare_walk(Run run)
{
    TableScope ts(kTablesPrepare);
    tables_missing() = false;
    const int rc = run();
    tables_missing() = false;
    return rc;
}

HDC_EXPORT int hdc_prepare(int dims, const int64_t* L, const int64_t* M, const int64_t* m, const int64_t* p,
                           const int64_t* q, const int64_t* D, int dtype, int64_t batch)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    return prepare_walk([&]() {
        return dtype == HDC_C128
                   ? conv_nd<double>(dims, no_data(0), no_data(1), (void*)no_data(2), ax, 0, batch, (void*)no_data(9), 0, nullptr)
                   : conv_nd<float>(dims, no_data(0), no_data(1), (void*)no_data(2), ax, 0, batch, (void*)no_data(9), 0, nullptr);
    });
}

HDC_EXPORT int hdc_prepare_window(int dims, const int64_t* L, const int64_t* M, const int64_t* m, const int64_t* p,
                                  const int64_t* q, const int64_t* D, const int64_t* o, const int64_t* Lw, int dtype,
                                  int64_t batch)
{
    if (!o || !Lw) return HDC_ERR_PARAM;
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax, o, Lw);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    return prepare_walk([&]() {
        return dtype == HDC_C128
                   ? conv_nd<double>(dims, no_data(0), no_data(1), (void*)no_data(2), ax, 0, batch, (void*)no_data(9), 0, nullptr)
                   : conv_nd<float>(dims, no_data(0), no_data(1), (void*)no_data(2), ax, 0, batch, (void*)no_data(9), 0, nullptr);
    });
}

HDC_EXPORT int hdc_prepare_hermitian(int64_t K, const int64_t* m, const int64_t* D, int dtype, int64_t batch)
{
    Axis ax, ay;
    int rc = herm_resolve_any(K, m, D, dtype, &ax, &ay);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    return prepare_walk([&]() {
        return hdc_conv2d_hermitian(no_data(0), no_data(1), (void*)no_data(2), K, m, D, dtype, batch,
                                    (void*)no_data(9), 0, nullptr);
    });
}

HDC_EXPORT int hdc_prepare_unequal(int dims, const int64_t* Lf, const int64_t* Lg, const int64_t* M, const int64_t* m,
                                   const int64_t* lam, const int64_t* D, const int64_t* o, const int64_t* Lw, int dtype,
                                   int64_t batch)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all_uneq(dims, Lf, Lg, M, m, lam, D, o, Lw, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    return prepare_walk([&]() {
        return dtype == HDC_C128
                   ? conv_nd<double>(dims, no_data(0), no_data(1), (void*)no_data(2), ax, 0, batch, (void*)no_data(9), 0, nullptr)
                   : conv_nd<float>(dims, no_data(0), no_data(1), (void*)no_data(2), ax, 0, batch, (void*)no_data(9), 0, nullptr);
    });
}

HDC_EXPORT int hdc_prepare_multi(int dims, int n, int op, const int64_t* L, const int64_t* M, const int64_t* m,
                                 const int64_t* p, const int64_t* q, const int64_t* D, int dtype, int64_t batch)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all_multi(dims, n, op, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    const void* xs[kMaxInputs];
    for (int i = 0; i < n; ++i) xs[i] = no_data(i);
    return prepare_walk([&]() {
        return dtype == HDC_C128
                   ? conv_nd_multi<double>(dims, n, op, xs, (void*)no_data(kMaxInputs), ax, batch, (void*)no_data(9), 0, nullptr)
                   : conv_nd_multi<float>(dims, n, op, xs, (void*)no_data(kMaxInputs), ax, batch, (void*)no_data(9), 0, nullptr);
    });
}

HDC_EXPORT int hdc_prepare_real(int dims, const int64_t* L, const int64_t* M, const int64_t* m, const int64_t* p,
                                const int64_t* q, const int64_t* D, int dtype, int64_t batch)
{
    Axis ax[HDC_MAX_DIMS];
    int rc = resolve_all(dims, L, M, m, p, q, D, dtype, ax);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    return prepare_walk([&]() {
        return dtype == HDC_C128
                   ? conv_nd_real<double>(dims, no_data(0), no_data(1), (void*)no_data(2), ax, batch, (void*)no_data(9), 0, nullptr)
                   : conv_nd_real<float>(dims, no_data(0), no_data(1), (void*)no_data(2), ax, batch, (void*)no_data(9), 0, nullptr);
    });
}

HDC_EXPORT int hdc_release_caches(void)
{
    std::lock_guard<std::mutex> lk(g_tw_mu);
    int rc = HDC_OK;
    for (auto& kv : g_tw) {
        int dev = std::get<0>(kv.first);
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(dev);
        if (cudaFree(kv.second) != cudaSuccess) rc = HDC_ERR_CUDA;
        cudaSetDevice(cur);
    }
    g_tw.clear();
    return rc;
}

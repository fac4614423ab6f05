// hdc_kernels.cu -- the CUDA kernels of the hot path and their launchers.
//
//  k_twiddle        zeta_n^k table in FP64 (exact integer angle, sincospi)
//  k_residue_rows   fused per (row, residue): fold (Eq. 1 inner sums) of f and
//                   g -> m-point FFTs -> pointwise product (Section 2.4) ->
//                   m-point inverse FFT (Eq. 2 inner sum); unscaled result
//  k_fold_fft_cols  fold along a strided axis + FFT over that axis, a tile of
//                   C neighbouring columns per block (N-D outer axes, and the
//                   first half of a split m = m1 m2 transform); the tile's
//                   fold blocks arrive by TMA box copies when the layout
//                   allows it
//  k_ifft_cols      inverse FFT over a strided axis, in place
//  k_unfold         twiddled unfold-accumulate of the first L outputs (Eq. 2
//                   outer sums), residues summed in increasing r, one scale
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <map>
#include <cudaTypedefs.h>
#include <mutex>

#include "hdc.h"
#include "hdc_bodies.cuh"
#include "hdc_internal.h"
#include "hdc_tma.cuh"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace hdc {

// First error a kernel of this file recorded instead of waiting forever
// (HDC_ERR_TIMEOUT); read and cleared by hdc_device_status.
__device__ int g_device_status = 0;

// TMA-staged loads in the strided fold (hdc_set_tma).
static std::atomic<int> g_fold_tma{ 1 };

static int sm_count();
template <typename T> static bool latency_launch(int64_t blocks);
static int latency_threads(int64_t elems);

// ------------------------------------------------------------- twiddles

template <class V>
__global__ void k_twiddle(V* tw, int64_t n)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    // angle 2 pi k / n folded into (-pi, pi] in integers, then one FP64
    // sincospi: the table entry is rounded once, never built by recurrence.
    const int64_t kk = (2 * k > n) ? k - n : k;
    double s, c;
    sincospi(2.0 * (double)kk / (double)n, &s, &c);
    using T = typename real_of<V>::type;
    tw[k] = mkc<V>((T)c, (T)s);
}

// The same values in scale-tangent form for the twiddle-merged butterflies:
// w = scale (1 + i t) with scale = cos, t = tan when |cos| >= |sin| (form 0),
// else w = i scale (1 + i t) with scale = sin, t = -cot (form 1); the form is
// stored in the last mantissa bit of scale (a change of one unit in the last
// place).
__device__ __forceinline__ void lf_store(double2* tw, int64_t k, double sc, double tt, int form)
{
    long long b = (__double_as_longlong(sc) & ~1LL) | (long long)form;
    tw[k] = make_double2(__longlong_as_double(b), tt);
}
__device__ __forceinline__ void lf_store(float2* tw, int64_t k, double sc, double tt, int form)
{
    int b = (__float_as_int((float)sc) & ~1) | form;
    tw[k] = make_float2(__int_as_float(b), (float)tt);
}

template <class V>
__global__ void k_twiddle_lf(V* tw, int64_t n)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t kk = (2 * k > n) ? k - n : k;
    double s, c;
    sincospi(2.0 * (double)kk / (double)n, &s, &c);
    if (fabs(c) >= fabs(s)) lf_store(tw, k, c, s / c, 0);
    else lf_store(tw, k, s, -c / s, 1);
}

template <typename T>
cudaError_t launch_twiddle_lf(cx<T>* tw, int64_t n, cudaStream_t st)
{
    const int thr = 256;
    const int64_t blocks = (n + thr - 1) / thr;
    LaunchScope ls(K_TWIDDLE, st, 0.0, (double)n * sizeof(cx<T>));
    k_twiddle_lf<cx<T>><<<(unsigned)blocks, thr, 0, st>>>(tw, n);
    return cudaGetLastError();
}
template cudaError_t launch_twiddle_lf<double>(cx<double>*, int64_t, cudaStream_t);
template cudaError_t launch_twiddle_lf<float>(cx<float>*, int64_t, cudaStream_t);

template <typename T>
cudaError_t launch_twiddle(cx<T>* tw, int64_t n, cudaStream_t st)
{
    const int thr = 256;
    const int64_t blocks = (n + thr - 1) / thr;
    LaunchScope ls(K_TWIDDLE, st, 0.0, (double)n * sizeof(cx<T>));
    k_twiddle<cx<T>><<<(unsigned)blocks, thr, 0, st>>>(tw, n);
    return cudaGetLastError();
}
template cudaError_t launch_twiddle<double>(cx<double>*, int64_t, cudaStream_t);
template cudaError_t launch_twiddle<float>(cx<float>*, int64_t, cudaStream_t);

// ------------------------------------------------------- helpers (host)

// One thread per radix-8 butterfly of the transform, within [64, kMaxThreads].
static int threads_for(int64_t elems)
{
    int64_t t = (elems + 7) / 8;
    t = ((t + 31) / 32) * 32;
    if (t < 64) t = 64;
    if (t > kMaxThreads) t = kMaxThreads;
    return (int)t;
}

// Opt a kernel in to `bytes` of dynamic shared memory when that passes the
// default limit, which is 48 KiB minus the kernel's static shared memory
// (the TMA fold's barrier, for one).  The limit each kernel already has is
// remembered, so a launch costs one lookup.
template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> granted; // (device, kernel) -> bytes allowed
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_pair(dev, reinterpret_cast<const void*>(kernel));
    std::lock_guard<std::mutex> lk(mu);
    auto it = granted.find(key);
    if (it != granted.end() && bytes <= it->second) return cudaSuccess;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return e;
    size_t limit = 48 * 1024 > fa.sharedSizeBytes ? 48 * 1024 - fa.sharedSizeBytes : 0;
    if (bytes > limit) {
        if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) != cudaSuccess)
            return e;
        limit = bytes;
    }
    granted[key] = it != granted.end() && it->second > limit ? it->second : limit;
    return cudaSuccess;
}

// ------------------------------------------------------- residue rows

template <class V, bool R16>
__global__ void __launch_bounds__(kMaxThreads, 2)
k_residue_rows(const V* f, const V* g, V* h, int64_t B, int64_t ld_f, int64_t ld_g, int64_t Lf, int64_t L, int m,
               int p, int q, int r0, int Dg, const TwTab<V> twN, const V* __restrict__ twm,
               const V* __restrict__ twml, FftPlan fp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int64_t b = blockIdx.x % B;
    const int rr = (int)(blockIdx.x / B);
    residue_row_body<V, R16>(f + b * ld_f, g + b * ld_g, h + ((int64_t)rr * B + b) * m, L, Lf, m, p, q, r0 + rr, twN,
                        twm, twml, fp, reinterpret_cast<V*>(smraw), threadIdx.x, blockDim.x);
}

template <typename T>
cudaError_t launch_residue_rows(const cx<T>* f, const cx<T>* g, cx<T>* h, int64_t B, int64_t ld_f, int64_t ld_g,
                                int64_t Lf, int64_t L, int64_t m, int64_t p, int64_t q, int64_t r0, int64_t D,
                                cudaStream_t st)
{
    using V = cx<T>;
    const int64_t Dg = (D < q - r0) ? D : (q - r0);
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const TwTab<V> twN = tw_table<T>(q * m, &e);
    if (e != cudaSuccess) return e;
    const bool lat = latency_launch<T>(B * Dg);
    const FftPlan fp = lat ? fft_plan_latency<T>(m) : fft_plan<T>(m, rows_r16(m));
    const V* twm = twiddles_fft_plan<T>(fp, false, &e);
    if (e != cudaSuccess) return e;
    const V* twml = twiddles_fft_plan<T>(fp, true, &e);
    if (e != cudaSuccess) return e;
    const int thr = lat ? latency_threads(m) : threads_for(m);
    const size_t smem = (size_t)(3 * smem_len<V>(m)) * sizeof(V);
    auto kern = takes_r16<V>(fp) ? k_residue_rows<V, kHas16<V>> : k_residue_rows<V, false>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    const int64_t blocks = B * Dg;
    // model: 3 FFTs + product per residue, and the fold of f and g (8 flops
    // per element each) unless the fold is a plain copy (p = q = 1)
    const double Lrow = (double)((L < p * m) ? L : p * m);
    const double Lfrow = (double)((Lf < p * m) ? Lf : p * m);
    const double fold = (p == 1 && q == 1 && Lf == L) ? 0.0 : 8.0 * (Lrow + Lfrow);
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_RESIDUE_ROWS, st, (double)(B * Dg) * (3.0 * fft_flops((double)m) + 6.0 * m + fold),
                   (B * (Lrow + Lfrow) + (double)(Dg * B * m)) * sizeof(V));
    kern<<<(unsigned)blocks, thr, smem, st>>>(f, g, h, B, ld_f, ld_g, Lf, L, (int)m, (int)p, (int)q, (int)r0,
                                              (int)Dg, twN, twm, twml, fp);
    return cudaGetLastError();
}

template <class V>
__global__ void __launch_bounds__(kMaxThreads, 2)
k_residue_rows_lam(const V* f, const V* g, V* h, int64_t B, int64_t ld_f, int64_t ld_g, int64_t Lf, int64_t Lg,
                   int mf, int lam, int pf, int pg, int qg, int r0, int Dg, const TwTab<V> twN,
                   const V* __restrict__ twf, const V* __restrict__ twfl, FftPlan fpf, const V* __restrict__ twg,
                   const V* __restrict__ twgl, FftPlan fpg)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int64_t b = blockIdx.x % B;
    const int rr = (int)(blockIdx.x / B);
    const int mg = mf * lam;
    residue_row_lam_body<V>(f + b * ld_f, g + b * ld_g, h + ((int64_t)rr * B + b) * mg, Lf, Lg, mf, mg, lam, pf, pg,
                            qg, r0 + rr, twN, twf, twfl, fpf, twg, twgl, fpg, reinterpret_cast<V*>(smraw),
                            threadIdx.x, blockDim.x);
}

template <typename T>
cudaError_t launch_residue_rows_lam(const cx<T>* f, const cx<T>* g, cx<T>* h, int64_t B, int64_t ld_f,
                                    int64_t ld_g, int64_t Lf, int64_t Lg, int64_t mf, int64_t lam, int64_t pf,
                                    int64_t pg, int64_t qg, int64_t r0, int64_t D, cudaStream_t st)
{
    using V = cx<T>;
    const int64_t Dg = (D < qg - r0) ? D : (qg - r0);
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    const int64_t mg = mf * lam;
    cudaError_t e = cudaSuccess;
    const TwTab<V> twN = tw_table<T>(qg * mg, &e);
    if (e != cudaSuccess) return e;
    const V* twf = twiddles_fft<T>(mf, false, &e);
    if (e != cudaSuccess) return e;
    const V* twfl = twiddles_fft<T>(mf, true, &e);
    if (e != cudaSuccess) return e;
    const V* twg = twiddles_fft<T>(mg, false, &e);
    if (e != cudaSuccess) return e;
    const V* twgl = twiddles_fft<T>(mg, true, &e);
    if (e != cudaSuccess) return e;
    const FftPlan fpf = fft_plan<T>(mf), fpg = fft_plan<T>(mg);
    const int thr = threads_for(mg);
    const size_t smem = (size_t)(3 * smem_len<V>(mg)) * sizeof(V);
    auto kern = k_residue_rows_lam<V>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    const int64_t blocks = B * Dg;
    // model per (row, residue of g): 2 mg-point FFTs, lam mf-point FFTs,
    // lam mf products, and the folds (8 flops per valid element per residue)
    const double Lgr = (double)((Lg < pg * mg) ? Lg : pg * mg);
    const double Lfr = (double)((Lf < pf * mf) ? Lf : pf * mf);
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_RESIDUE_ROWS, st,
                   (double)(B * Dg) * (2.0 * fft_flops((double)mg) + lam * fft_flops((double)mf) + 6.0 * mg +
                                       8.0 * (Lgr + lam * Lfr)),
                   (B * (Lgr + Lfr) + (double)(Dg * B * mg)) * sizeof(V));
    kern<<<(unsigned)blocks, thr, smem, st>>>(f, g, h, B, ld_f, ld_g, Lf, Lg, (int)mf, (int)lam, (int)pf, (int)pg,
                                              (int)qg, (int)r0, (int)Dg, twN, twf, twfl, fpf, twg, twgl, fpg);
    return cudaGetLastError();
}

template <class V>
__global__ void __launch_bounds__(kMaxThreads, 2)
k_residue_rows_multi(InPtrs<V> in, int nin, int op, V* h, int64_t B, int64_t ld, int64_t L, int m, int p, int q,
                     int r0, int Dg, const TwTab<V> twN, const V* __restrict__ twm,
                     const V* __restrict__ twml, FftPlan fp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int64_t b = blockIdx.x % B;
    const int rr = (int)(blockIdx.x / B);
    residue_row_multi_body<V>(in, nin, op, b * ld, h + ((int64_t)rr * B + b) * m, L, m, p, q, r0 + rr, twN, twm,
                              twml, fp, reinterpret_cast<V*>(smraw), threadIdx.x, blockDim.x);
}

template <typename T>
cudaError_t launch_residue_rows_multi(const cx<T>* const* xs, int nin, int op, cx<T>* h, int64_t B, int64_t ld,
                                      int64_t L, int64_t m, int64_t p, int64_t q, int64_t r0, int64_t D,
                                      cudaStream_t st)
{
    using V = cx<T>;
    if (nin < 1 || nin > kMaxInputs || op < 0 || op > 1 || (op == 1 && (nin & 1))) return cudaErrorInvalidValue;
    const int64_t Dg = (D < q - r0) ? D : (q - r0);
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const TwTab<V> twN = tw_table<T>(q * m, &e);
    if (e != cudaSuccess) return e;
    const V* twm = twiddles_fft<T>(m, false, &e);
    if (e != cudaSuccess) return e;
    const V* twml = twiddles_fft<T>(m, true, &e);
    if (e != cudaSuccess) return e;
    const FftPlan fp = fft_plan<T>(m);
    const int thr = threads_for(m);
    const size_t smem = (size_t)(3 * smem_len<V>(m)) * sizeof(V);
    auto kern = k_residue_rows_multi<V>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    InPtrs<V> in;
    for (int i = 0; i < kMaxInputs; ++i) in.x[i] = xs[i < nin ? i : 0];
    const int64_t blocks = B * Dg;
    // model: nin forward FFTs, one inverse, nin - 1 products (op 0) or
    // nin / 2 products and nin / 2 - 1 sums (op 1), the folds
    const double Lrow = (double)((L < p * m) ? L : p * m);
    const double fold = (p == 1 && q == 1) ? 0.0 : 8.0 * nin * Lrow;
    const double pointwise = op == 0 ? 6.0 * (nin - 1) * m : (6.0 * (nin / 2) + 2.0 * (nin / 2 - 1)) * m;
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_RESIDUE_ROWS, st, (double)(B * Dg) * ((nin + 1.0) * fft_flops((double)m) + pointwise + fold),
                   (nin * B * Lrow + (double)(Dg * B * m)) * sizeof(V));
    kern<<<(unsigned)blocks, thr, smem, st>>>(in, nin, op, h, B, ld, L, (int)m, (int)p, (int)q, (int)r0, (int)Dg,
                                              twN, twm, twml, fp);
    return cudaGetLastError();
}

// ------------------------------------------------ strided-axis passes

// Blocks per SM the column kernels are compiled for: three in FP32, whose
// passes wait on memory and want the extra warps; two in FP64, whose
// transforms want the registers.
template <class V> constexpr int kColBlocks = sizeof(V) == 8 ? 3 : 2;

// SMs of the current device (asked once per device and remembered).
static int sm_count()
{
    constexpr int kDevs = 64;
    static std::atomic<int> known[kDevs];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) return 152;
    int sms = known[dev].load();
    if (sms > 0) return sms;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    known[dev].store(sms);
    return sms;
}

// An FP64 launch of at most two waves (two blocks per SM) waits on the
// serial FFT stages of its blocks rather than on the FP64 pipe's throughput:
// it takes the radix-2 latency plan (fft_plan_latency: the same FMAs per
// point, spread over four times the threads) and one thread per radix-2
// butterfly of a stage, up to kMaxThreads.  Larger launches keep radix 8.
template <typename T> static bool latency_launch(int64_t blocks)
{
    return sizeof(T) == 8 && blocks <= 4 * (int64_t)sm_count();
}
static int latency_threads(int64_t elems)
{
    int64_t t = (elems / 2 + 31) / 32 * 32;
    if (t < 64) t = 64;
    if (t > kMaxThreads) t = kMaxThreads;
    return (int)t;
}

// Column tile width C.  FP32 passes wait on memory: the widest power of two
// up to 256 whose tile (ma C elements) fits elems_max, narrowed (down to 16)
// while the launch would have fewer than four blocks per SM (`others` blocks
// per tile position).  FP64 passes are bound by their arithmetic and run
// best in small blocks: 16 columns, or as many as give a short axis (ma <
// 32) 512 elements, i.e. 64 threads of work.  Never wider than the columns
// need.
template <typename T> static int col_tile(int64_t Cn, int64_t ma, int64_t elems_max, int64_t others)
{
    int64_t C = 256;
    if (sizeof(T) == 8) {
        int64_t c16 = 16;
        while (c16 < 256 && ma * c16 < 512) c16 <<= 1;
        C = c16;
    }
    while (C > 1 && ma * C > elems_max) C >>= 1;
    if (sizeof(T) == 4) {
        const int64_t want = 4 * (int64_t)sm_count();
        while (C > 16 && others * ((Cn + C - 1) / C) < want) C >>= 1;
    }
    while (C > 1 && C / 2 >= Cn) C >>= 1;
    return (int)C;
}

template <class V> struct ColSideK {
    const V* x;
    V* y;
    int64_t bstride, Lvalid;
    int p, q, rmul, lam, rneg;
};
template <class V> struct ColSidesK {
    ColSideK<V> s[kMaxInputs];
};

// One tensor map per input of the strided fold: x[b][a][c] as 8-byte units,
// dims (Cn * sizeof(V) / 8, full rows, B), box (C columns, tma_rows rows, 1).
struct ColMapsK {
    CUtensorMap m[kMaxInputs];
};

// Give up on a copy after about a second of SM clocks.
constexpr long long kTmaWaitCycles = 2000000000LL;

// Fold of the tile's p <= 2 blocks from the TMA-staged copies: block t of
// the tile (rows t ma .. t ma + ma - 1) was copied to buf + t * stride as far
// as it holds full rows of x (a < afull = Lvalid / Cn); the partial row
// a = afull (when Lvalid is not a multiple of Cn) is read here with plain
// loads and the rows past it are zero.  The folded tile goes to buf.
template <class V>
__device__ __forceinline__ void fold_staged_tile(V* buf, int stride, const V* x, int64_t Cn, int ma, int p, int q,
                                                 int64_t Nf, int64_t cs, int64_t cc, int64_t Lvalid, int r,
                                                 int64_t c0, int C, const TwTab<V> twNf, int tid, int nthr)
{
    const int64_t mq = Nf / q;
    const int64_t afull = Lvalid / Cn;
    const int n = ma * C;
    for (int e = tid; e < n; e += nthr) {
        const int i = div_idx(e, C), cl = e - i * C;
        const int64_t c = c0 + cl;
        V acc = czero<V>();
        for (int t = 0; t < p; ++t) {
            const int64_t a = (int64_t)t * ma + i;
            V v = czero<V>();
            if (a < afull) v = buf[t * stride + e];
            else if (a == afull && c < Cn && a * Cn + c < Lvalid) v = x[a * Cn + c];
            // block t = 0 carries zeta_q^0 = 1: no multiplication
            if (t == 0) acc = v;
            else if (r == 0) acc = cadd(acc, v);
            else acc = cfma(v, twn(twNf, rt_mod(r, t, q) * mq), acc);
        }
        if (r != 0 && c < Cn) acc = cmul(acc, twn(twNf, (int64_t)r * (i * cs + c * cc)));
        buf[e] = acc;
    }
}

// The block of the strided fold: column tile ct, input `which`, residue
// block (l, rr) of batch row b; residue r, input row x, output yb.  skip: a
// self-paired residue's partner, whose column pass the other side does.
template <class V> struct FoldBlock {
    int which, r, skip;
    int64_t b, c0;
    const V* x;
    V* yb;
};

template <class V>
__device__ __forceinline__ FoldBlock<V> fold_block(const ColSidesK<V>& sides, int nside, int64_t B, int64_t Cn, int ma,
                                                   int r0, int Dg, int C, int nct)
{
    FoldBlock<V> fb;
    int64_t blk = blockIdx.x;
    const int ct = (int)(blk % nct);
    blk /= nct;
    fb.which = (int)(blk % nside);
    blk /= nside;
    const ColSideK<V>& sd = sides.s[fb.which];
    const int nres = Dg * sd.lam;
    const int rt = (int)(blk % nres);
    fb.b = blk / nres;
    const int l = rt / Dg, rr = rt - l * Dg;
    fb.x = sd.x + fb.b * sd.bstride;
    fb.yb = sd.y + ((int64_t)rr * B + fb.b) * ((int64_t)ma * sd.lam) * Cn + (int64_t)l * Cn;
    fb.r = sd.rneg ? (sd.q - (r0 + rr)) % sd.q : r0 + rr + l * sd.rmul;
    fb.skip = sd.rneg && fb.r == r0 + rr;
    fb.c0 = (int64_t)ct * C;
    return fb;
}

template <class V, bool R16>
__global__ void __launch_bounds__(kMaxThreads, kColBlocks<V>)
k_fold_fft_cols(ColSidesK<V> sides, int nside, int64_t B, int64_t Cn, int ma, int64_t Nf, int64_t cs, int64_t cc,
                int r0, int Dg, int C, int nct, int post, const TwTab<V> twNf, const V* __restrict__ tpm,
                const V* __restrict__ twma, const V* __restrict__ twmal, FftPlan fp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const FoldBlock<V> fb = fold_block<V>(sides, nside, B, Cn, ma, r0, Dg, C, nct);
    // (the whole block leaves before any barrier)
    if (fb.skip) return;
    const ColSideK<V>& sd = sides.s[fb.which];
    fold_fft_cols_body<V, R16>(fb.x, fb.yb, Cn, ma, sd.p, sd.q, Nf, cs, cc, sd.Lvalid, fb.r, fb.c0, C, post,
                          (int64_t)sd.lam * Cn, twNf, tpm, twma, twmal, fp, reinterpret_cast<V*>(smraw), threadIdx.x,
                          blockDim.x);
}

// The same pass with the tile's fold blocks staged by TMA box copies of
// tma_rows rows (the host has checked every copy rule; a block whose shared
// memory is not 128-byte aligned uses the plain loads).
template <class V, bool R16>
__global__ void __launch_bounds__(kMaxThreads, kColBlocks<V>)
k_fold_fft_cols_tma(ColSidesK<V> sides, const __grid_constant__ ColMapsK maps, int tma_rows, int nside, int64_t B,
                    int64_t Cn, int ma, int64_t Nf, int64_t cs, int64_t cc, int r0, int Dg, int C, int nct, int post,
                    const TwTab<V> twNf, const V* __restrict__ tpm, const V* __restrict__ twma,
                    const V* __restrict__ twmal, FftPlan fp)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ uint64_t bar;
    const FoldBlock<V> fb = fold_block<V>(sides, nside, B, Cn, ma, r0, Dg, C, nct);
    if (fb.skip) return;
    const ColSideK<V>& sd = sides.s[fb.which];
    V* buf = reinterpret_cast<V*>(smraw);
    const int tid = threadIdx.x, nthr = blockDim.x;
    if ((smem_u32(buf) & 127) != 0) {
        fold_fft_cols_body<V, R16>(fb.x, fb.yb, Cn, ma, sd.p, sd.q, Nf, cs, cc, sd.Lvalid, fb.r, fb.c0, C, post,
                              (int64_t)sd.lam * Cn, twNf, tpm, twma, twmal, fp, buf, tid, nthr);
        return;
    }
    const int n = ma * C;
    const int stride = (int)smem_len<V>(n);
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        // boxes that start past the last full row are not copied (their rows
        // are zero or the partial row); a box that runs past it is filled
        // with zeros there and still delivers all its bytes
        constexpr int kUnits = (int)(sizeof(V) / 8);
        const int64_t afull = sd.Lvalid / Cn;
        uint32_t nbox = 0;
        for (int t = 0; t < sd.p; ++t)
            for (int j = 0; j * tma_rows < ma; ++j) nbox += (int64_t)t * ma + j * tma_rows < afull;
        mbar_arrive_expect_tx(&bar, nbox * (uint32_t)(tma_rows * C * sizeof(V)));
        for (int t = 0; t < sd.p; ++t)
            for (int j = 0; j * tma_rows < ma; ++j)
                if ((int64_t)t * ma + j * tma_rows < afull)
                    tma_load_3d(buf + t * stride + j * tma_rows * C, &maps.m[fb.which], (int)(fb.c0 * kUnits),
                                t * ma + j * tma_rows, (int)fb.b, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, kTmaWaitCycles);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicCAS(&g_device_status, 0, (int)HDC_ERR_TIMEOUT);
        return;
    }
    fold_staged_tile<V>(buf, stride, fb.x, Cn, ma, sd.p, sd.q, Nf, cs, cc, sd.Lvalid, fb.r, fb.c0, C, twNf, tid,
                        nthr);
    __syncthreads();
    fft_cols_store_body<V, R16>(buf, buf + stride, fb.yb, Cn, ma, sd.q, fb.c0, C, post, (int64_t)sd.lam * Cn, twNf, tpm,
                           twma, twmal, fp, tid, nthr);
}

// The column-major four-step twiddle table of an FP64 ma x Cn split when a
// pass applies those twiddles (flag set and Nf / q = ma Cn), else null (the
// kernels then read zeta_{Nf/q}^{l c} from the fold/unfold table).  FP32
// reads its large fold tables as two small ones (TwTab), which measured
// faster than this m-entry table (2^22: 6 % slower with it); FP64 gains
// 1-4 % with it.
template <typename T>
static const cx<T>* fourstep_table(int flag, int64_t Nf, int64_t q, int64_t ma, int64_t Cn, cudaError_t* e)
{
    if (sizeof(T) != 8 || !flag || q <= 0 || Nf % q != 0 || Nf / q != ma * Cn) return nullptr;
    return twiddles_colmajor<T>(ma, Cn, e);
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on it);
// null if the driver does not offer it.
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Rows per TMA box for a tile of ma rows x C columns of es-byte elements: a
// divisor of ma of at most 256 (the box limit) such that every box starts
// 128-byte aligned in shared memory; 0 if none of at least 8 rows exists.
static int tma_box_rows(int64_t ma, int64_t C, int64_t es)
{
    for (int64_t d = ma < 256 ? ma : 256; d >= 8; --d)
        if (ma % d == 0 && (d == ma || (d * C * es) % 128 == 0)) return (int)d;
    return ma < 8 ? (int)ma : 0;
}

// Tensor maps for the TMA-staged fold of every input, or 0 when one of them
// does not meet the copy rules (then the plain loads are used).  Returns the
// rows per box.
template <class V>
static int make_fold_maps(ColMapsK* maps, const ColSidesK<V>& k, int nside, int64_t B, int64_t Cn, int64_t ma,
                          int C)
{
    const int64_t es = (int64_t)sizeof(V);
    const int64_t units = es / 8;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc || C * units > 256 || (C * es) % 16 != 0 || (Cn * es) % 16 != 0) return 0;
    const int rows = tma_box_rows(ma, C, es);
    if (rows == 0) return 0;
    // the boxes the kernel issues, checked here: each destination 128-byte
    // aligned inside its block's half of the 2 smem_len(ma C) buffer, the
    // bytes one barrier expects below its 2^20 limit
    const int64_t n = ma * C, stride = smem_len<V>(n);
    if (ma % rows != 0 || (stride * es) % 128 != 0 || 2 * n * es >= ((int64_t)1 << 20)) return 0;
    for (int64_t j = 0; j * rows < ma; ++j)
        if ((j * rows * C * es) % 128 != 0 || (j + 1) * rows * C > n) return 0;
    for (int i = 0; i < nside; ++i) {
        const ColSideK<V>& sd = k.s[i];
        const int64_t afull = sd.Lvalid / Cn;
        if (sd.p > 2 || afull < 1 || ((uintptr_t)sd.x % 16) != 0) return 0;
        if (B > 1 && (sd.bstride * es) % 16 != 0) return 0;
        if (afull > ((int64_t)1 << 31) || Cn * units > ((int64_t)1 << 31) || B > ((int64_t)1 << 31)) return 0;
        const cuuint64_t dims[3] = { (cuuint64_t)(Cn * units), (cuuint64_t)afull, (cuuint64_t)B };
        const int64_t bs = B > 1 ? sd.bstride * es : (afull * Cn * es + 15) / 16 * 16;
        const cuuint64_t strides[2] = { (cuuint64_t)(Cn * es), (cuuint64_t)bs };
        const cuuint32_t box[3] = { (cuuint32_t)(C * units), (cuuint32_t)rows, 1 };
        const cuuint32_t estr[3] = { 1, 1, 1 };
        if (enc(&maps->m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, (void*)sd.x, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return 0;
    }
    return rows;
}

template <typename T>
cudaError_t launch_fold_fft_cols(const ColSide<T>* sides, int nside, int64_t B, int64_t Cn, int64_t ma, int64_t Nf,
                                 int64_t cs, int64_t cc, int64_t r0, int64_t D, int post, cudaStream_t st)
{
    using V = cx<T>;
    if (nside < 1 || nside > kMaxInputs) return cudaErrorInvalidValue;
    for (int i = 0; i < nside && nside > 1; ++i)
        if (sides[i].lam != 1) return cudaErrorInvalidValue;
    const int64_t q0 = sides[nside - 1].q;
    const int64_t Dg = (D < q0 - r0) ? D : (q0 - r0);
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const TwTab<V> twNf = tw_table<T>(Nf, &e);
    if (e != cudaSuccess) return e;
    const int Cw = col_tile<T>(Cn, ma, col_tile_target<T>(), Dg * sides[0].lam * nside * B);
    const bool lat = latency_launch<T>(((Cn + Cw - 1) / Cw) * Dg * sides[0].lam * nside * B);
    const FftPlan fp = lat ? fft_plan_latency<T>(ma) : fft_plan<T>(ma, true);
    const V* twma = twiddles_fft_plan<T>(fp, false, &e);
    if (e != cudaSuccess) return e;
    const V* twmal = twiddles_fft_plan<T>(fp, true, &e);
    if (e != cudaSuccess) return e;
    bool same_q = true;
    for (int i = 1; i < nside; ++i) same_q = same_q && sides[i].q == sides[0].q && sides[i].lam == 1;
    const V* tpm = (same_q && sides[0].lam == 1) ? fourstep_table<T>(post, Nf, q0, ma, Cn, &e) : nullptr;
    if (e != cudaSuccess) return e;
    const int C = Cw;
    const int nct = (int)((Cn + C - 1) / C);
    const int thr = lat ? latency_threads(ma * C) : threads_for(ma * C);
    const size_t smem = (size_t)(2 * smem_len<V>(ma * C)) * sizeof(V);
    ColSidesK<V> k;
    double flops = 0.0, bytes = 0.0;
    for (int i = 0; i < kMaxInputs; ++i) {
        const ColSide<T>& sd = sides[i < nside ? i : 0];
        k.s[i] = ColSideK<V>{ sd.x, sd.y, sd.bstride, sd.Lvalid, sd.p, sd.q, sd.rmul, sd.lam, sd.rneg };
        if (i < nside) {
            flops += (double)Dg * sd.lam * B * (8.0 * sd.Lvalid + (double)Cn * fft_flops((double)ma));
            bytes += (B * (double)sd.Lvalid + (double)Dg * sd.lam * B * ma * Cn) * sizeof(V);
        }
    }
    const int64_t blocks = (int64_t)nct * Dg * sides[0].lam * nside * B;
    if (preparing()) return cudaSuccess; // the walk of hdc_prepare*: tables made, nothing launched
    ColMapsK maps;
    memset(&maps, 0, sizeof maps);
    const int tma_rows = g_fold_tma ? make_fold_maps<V>(&maps, k, nside, B, Cn, ma, C) : 0;
    if (tma_rows > 0) {
        auto kern = takes_r16<V>(fp) ? k_fold_fft_cols_tma<V, kHas16<V>> : k_fold_fft_cols_tma<V, false>;
        if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
        LaunchScope ls(K_FOLD_TMA, st, flops, bytes);
        kern<<<(unsigned)blocks, thr, smem, st>>>(k, maps, tma_rows, nside, B, Cn, (int)ma, Nf, cs, cc, (int)r0,
                                                  (int)Dg, C, nct, post, twNf, tpm, twma, twmal, fp);
        return cudaGetLastError();
    }
    auto kern = takes_r16<V>(fp) ? k_fold_fft_cols<V, kHas16<V>> : k_fold_fft_cols<V, false>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    LaunchScope ls(K_FOLD_FFT_COLS, st, flops, bytes);
    kern<<<(unsigned)blocks, thr, smem, st>>>(k, nside, B, Cn, (int)ma, Nf, cs, cc, (int)r0, (int)Dg, C, nct, post,
                                              twNf, tpm, twma, twmal, fp);
    return cudaGetLastError();
}

template <class V, bool R16>
__global__ void __launch_bounds__(kMaxThreads, kColBlocks<V>)
k_ifft_cols(V* y, int64_t B, int64_t Cn, int ma, int q, int64_t Nf, int Dg, int C, int nct, int pre,
            const TwTab<V> twNf, const V* __restrict__ tpm, const V* __restrict__ twma, const V* __restrict__ twmal,
            FftPlan fp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    int64_t blk = blockIdx.x;
    const int ct = (int)(blk % nct);
    blk /= nct;
    const int rr = (int)(blk % Dg);
    const int64_t b = blk / Dg;
    ifft_cols_body<V, R16>(y + ((int64_t)rr * B + b) * ma * Cn, Cn, ma, q, Nf, (int64_t)ct * C, C, pre, twNf, tpm, twma,
                      twmal, fp, reinterpret_cast<V*>(smraw), threadIdx.x, blockDim.x);
}

template <typename T>
cudaError_t launch_ifft_cols(cx<T>* y, int64_t B, int64_t Cn, int64_t ma, int64_t q, int64_t Nf,
                             int64_t D, int pre, cudaStream_t st)
{
    using V = cx<T>;
    if (B <= 0 || D <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const TwTab<V> twNf = tw_table<T>(Nf, &e);
    if (e != cudaSuccess) return e;
    const int C = col_tile<T>(Cn, ma, col_tile_target<T>(), D * B);
    const int nct = (int)((Cn + C - 1) / C);
    const bool lat = latency_launch<T>((int64_t)nct * D * B);
    const FftPlan fp = lat ? fft_plan_latency<T>(ma) : fft_plan<T>(ma, true);
    const V* twma = twiddles_fft_plan<T>(fp, false, &e);
    if (e != cudaSuccess) return e;
    const V* twmal = twiddles_fft_plan<T>(fp, true, &e);
    if (e != cudaSuccess) return e;
    const V* tpm = fourstep_table<T>(pre, Nf, q, ma, Cn, &e);
    if (e != cudaSuccess) return e;
    const int thr = lat ? latency_threads(ma * C) : threads_for(ma * C);
    const size_t smem = (size_t)(2 * smem_len<V>(ma * C)) * sizeof(V);
    auto kern = takes_r16<V>(fp) ? k_ifft_cols<V, kHas16<V>> : k_ifft_cols<V, false>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    const int64_t blocks = (int64_t)nct * D * B;
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_IFFT_COLS, st, (double)(D * B) * (double)Cn * fft_flops((double)ma),
                   2.0 * D * B * ma * Cn * sizeof(V));
    kern<<<(unsigned)blocks, thr, smem, st>>>(y, B, Cn, (int)ma, (int)q, Nf, (int)D, C, nct, pre, twNf,
                                              tpm, twma, twmal, fp);
    return cudaGetLastError();
}

// --------------------------------------------------------------- unfold

template <class V, int PT>
__global__ void __launch_bounds__(256)
k_unfold(V* out, const V* __restrict__ h, int64_t B, int64_t bstride, int64_t Cn, int64_t ma,
         int p, int q, int64_t Nf, int64_t cs, int64_t cc, int64_t lo, int64_t hi, int r0, int Dg,
         int first, int last, typename real_of<V>::type scale, const TwTab<V> twNf)
{
    const int64_t per = ma * Cn;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= per * B) return;
    const int64_t b = div_idx(gid, per);
    const int64_t e = gid - b * per;
    const int64_t i = div_idx(e, Cn), c = e - i * Cn;
    unfold_elem<V, PT>(out + b * bstride, h + b * per, B * per, Cn, ma, i, c, p, q, Nf, cs, cc, lo, hi, r0, Dg,
                       first, last, scale, twNf);
}

template <typename T>
cudaError_t launch_unfold(cx<T>* out, const cx<T>* h, int64_t B, int64_t bstride, int64_t Cn,
                          int64_t ma, int64_t p, int64_t q, int64_t Nf, int64_t cs, int64_t cc,
                          int64_t lo, int64_t hi, int64_t r0, int64_t D, int first, int last, double scale,
                          cudaStream_t st)
{
    using V = cx<T>;
    const int64_t Dg = (D < q - r0) ? D : (q - r0);
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const TwTab<V> twNf = tw_table<T>(Nf, &e);
    if (e != cudaSuccess) return e;
    const int thr = 256;
    const int64_t total = ma * Cn * B;
    const int64_t blocks = (total + thr - 1) / thr;
    const double nout = (double)(hi - lo);
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_UNFOLD, st, (double)(Dg * B) * 8.0 * nout + (last ? 2.0 * B * nout : 0.0),
                   ((double)(Dg * B * ma * Cn) + (first ? 1.0 : 2.0) * B * nout) * sizeof(V));
    k_unfold<V, 4><<<(unsigned)blocks, thr, 0, st>>>(out, h, B, bstride, Cn, ma, (int)p, (int)q, Nf,
                                                     cs, cc, lo, hi, (int)r0, (int)Dg, first, last,
                                                     (T)scale, twNf);
    return cudaGetLastError();
}

// ------------------------------------------ inverse + unfold, fused

template <class V, bool R16>
__global__ void __launch_bounds__(kMaxThreads, kColBlocks<V>)
k_ifft_unfold_cols(const V* y, V* out, int64_t B, int64_t bstride, int64_t Cn, int ma, int p, int q, int64_t Nf,
                   int64_t cs, int64_t cc, int64_t lo, int64_t hi, int r0, int Dg, int first, int last,
                   typename real_of<V>::type scale, int C, int nct, int pre, const TwTab<V> twNf,
                   const V* __restrict__ tpm, const V* __restrict__ twma, const V* __restrict__ twmal, FftPlan fp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    int64_t blk = blockIdx.x;
    const int ct = (int)(blk % nct);
    const int64_t b = blk / nct;
    const int64_t per = (int64_t)ma * Cn;
    ifft_unfold_cols_body<V, R16>(y + b * per, B * per, out + b * bstride, Cn, ma, p, q, Nf, cs, cc, lo, hi, r0, Dg,
                             first, last, scale, (int64_t)ct * C, C, pre, twNf, tpm, twma, twmal, fp,
                             reinterpret_cast<V*>(smraw), threadIdx.x, blockDim.x);
}

template <typename T>
cudaError_t launch_ifft_unfold(cx<T>* y, cx<T>* out, int64_t B, int64_t bstride, int64_t Cn, int64_t ma, int64_t p,
                               int64_t q, int64_t Nf, int64_t cs, int64_t cc, int64_t lo, int64_t hi, int64_t r0,
                               int64_t D, int first, int last, double scale, int pre, cudaStream_t st)
{
    using V = cx<T>;
    const int64_t Dg = (D < q - r0) ? D : (q - r0);
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    const int C = col_tile<T>(Cn, ma, col_tile_target<T>(), B);
    const int nct = (int)((Cn + C - 1) / C);
    const int sms = sm_count();
    // with several residues per pass the fused form has D times fewer blocks
    // and re-reads its outputs once per residue: measured slower than the two
    // passes, so it is taken for one residue per pass only
    if (Dg != 1 || B * nct < 2 * (int64_t)sms) {
        cudaError_t e = launch_ifft_cols<T>(y, B, Cn, ma, q, Nf, Dg, pre, st);
        if (e != cudaSuccess) return e;
        return launch_unfold<T>(out, y, B, bstride, Cn, ma, p, q, Nf, cs, cc, lo, hi, r0, Dg, first, last, scale, st);
    }
    cudaError_t e = cudaSuccess;
    const TwTab<V> twNf = tw_table<T>(Nf, &e);
    if (e != cudaSuccess) return e;
    const bool lat = latency_launch<T>(B * nct);
    const FftPlan fp = lat ? fft_plan_latency<T>(ma) : fft_plan<T>(ma, true);
    const V* twma = twiddles_fft_plan<T>(fp, false, &e);
    if (e != cudaSuccess) return e;
    const V* twmal = twiddles_fft_plan<T>(fp, true, &e);
    if (e != cudaSuccess) return e;
    const V* tpm = fourstep_table<T>(pre, Nf, q, ma, Cn, &e);
    if (e != cudaSuccess) return e;
    const int thr = lat ? latency_threads(ma * C) : threads_for(ma * C);
    const size_t smem = (size_t)(2 * smem_len<V>(ma * C)) * sizeof(V);
    auto kern = takes_r16<V>(fp) ? k_ifft_unfold_cols<V, kHas16<V>> : k_ifft_unfold_cols<V, false>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    const double nout = (double)(hi - lo);
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_IFFT_UNFOLD, st,
                   (double)(Dg * B) * ((double)Cn * fft_flops((double)ma) + 8.0 * nout) + (last ? 2.0 * B * nout : 0.0),
                   ((double)(Dg * B * ma * Cn) + (first ? 1.0 : 2.0) * B * nout) * sizeof(V));
    kern<<<(unsigned)(B * nct), thr, smem, st>>>(y, out, B, bstride, Cn, (int)ma, (int)p, (int)q, Nf, cs, cc, lo, hi,
                                                 (int)r0, (int)Dg, first, last, (T)scale, C, nct, pre, twNf, tpm,
                                                 twma, twmal, fp);
    return cudaGetLastError();
}

// ------------------------------------------------------- real inputs

template <typename T> __global__ void k_pack_real(const T* __restrict__ f, const T* __restrict__ g, cx<T>* z, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) z[i] = mkc<cx<T>>(f[i], g[i]);
}

template <typename T> cudaError_t launch_pack_real(const T* f, const T* g, cx<T>* z, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int thr = 256;
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_UNFOLD, st, 0.0, (double)n * (2.0 * sizeof(T) + sizeof(cx<T>)));
    k_pack_real<T><<<(unsigned)((n + thr - 1) / thr), thr, 0, st>>>(f, g, z, n);
    return cudaGetLastError();
}

template <class V>
__global__ void __launch_bounds__(kMaxThreads, 2)
k_residue_rows_real(const V* z, V* h, int64_t B, int64_t ld, int64_t L, int m, int p, int q, int r0,
                    const TwTab<V> twN, const V* __restrict__ twm, const V* __restrict__ twml, FftPlan fp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int64_t b = blockIdx.x % B;
    const int rr = (int)(blockIdx.x / B);
    residue_row_real_body<V>(z + b * ld, h + ((int64_t)rr * B + b) * m, L, m, p, q, r0 + rr, twN, twm, twml, fp,
                             reinterpret_cast<V*>(smraw), threadIdx.x, blockDim.x);
}

template <typename T>
cudaError_t launch_residue_rows_real(const cx<T>* z, cx<T>* h, int64_t B, int64_t ld, int64_t L, int64_t m,
                                     int64_t p, int64_t q, int64_t r0, int64_t Dg, cudaStream_t st)
{
    using V = cx<T>;
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const TwTab<V> twN = tw_table<T>(q * m, &e);
    if (e != cudaSuccess) return e;
    const V* twm = twiddles_fft<T>(m, false, &e);
    if (e != cudaSuccess) return e;
    const V* twml = twiddles_fft<T>(m, true, &e);
    if (e != cudaSuccess) return e;
    const FftPlan fp = fft_plan<T>(m);
    const int thr = threads_for(m);
    const size_t smem = (size_t)(3 * smem_len<V>(m)) * sizeof(V);
    auto kern = k_residue_rows_real<V>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    // model per kept residue: two forward FFTs (one when self-paired, counted
    // as two), one inverse, the pair product, the folds of z
    const double Lrow = (double)((L < p * m) ? L : p * m);
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_RESIDUE_ROWS, st, (double)(B * Dg) * (3.0 * fft_flops((double)m) + 14.0 * m + 16.0 * Lrow),
                   (B * Lrow + (double)(Dg * B * m)) * sizeof(V));
    kern<<<(unsigned)(B * Dg), thr, smem, st>>>(z, h, B, ld, L, (int)m, (int)p, (int)q, (int)r0, twN, twm, twml, fp);
    return cudaGetLastError();
}

// Split route rows, real inputs: block (rr, b, l1) pairs row l1 of ya[rr][b]
// with row l1' of yb[rr][b] (of ya[rr][b] for a self-paired residue;
// l1' = (m1 - l1) mod m1 for residue 0, else m1 - 1 - l1) and writes row l1
// of yh[rr][b], which must not alias ya or yb; rows of m2.
template <class V>
__global__ void __launch_bounds__(kMaxThreads, 2)
k_rows_real_pair(const V* ya, const V* yb, V* yh, int64_t B, int m1, int m2, int q, int r0,
                 const V* __restrict__ twm, const V* __restrict__ twml, FftPlan fp)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    int64_t blk = blockIdx.x;
    const int l1 = (int)(blk % m1);
    blk /= m1;
    const int64_t b = blk % B;
    const int rr = (int)(blk / B);
    const int r = r0 + rr;
    const int l1p = r == 0 ? (m1 - l1) % m1 : m1 - 1 - l1;
    const int64_t base = ((int64_t)rr * B + b) * m1;
    // self-paired residues (r = 0, 2 r = q) find their partner rows in ya
    const V* src = (r == 0 || 2 * r == q) ? ya : yb;
    rows_real_pair_body<V>(ya + (base + l1) * m2, src + (base + l1p) * m2, yh + (base + l1) * m2, m2, r, l1, twm,
                           twml, fp, reinterpret_cast<V*>(smraw), threadIdx.x, blockDim.x);
}

template <typename T>
cudaError_t launch_rows_real_pair(const cx<T>* ya, const cx<T>* yb, cx<T>* yh, int64_t B, int64_t m1, int64_t m2,
                                  int64_t q, int64_t r0, int64_t Dg, cudaStream_t st)
{
    using V = cx<T>;
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const V* twm = twiddles_fft<T>(m2, false, &e);
    if (e != cudaSuccess) return e;
    const V* twml = twiddles_fft<T>(m2, true, &e);
    if (e != cudaSuccess) return e;
    const FftPlan fp = fft_plan<T>(m2);
    const int thr = threads_for(m2);
    const size_t smem = (size_t)(3 * smem_len<V>(m2)) * sizeof(V);
    auto kern = k_rows_real_pair<V>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    const int64_t rows = Dg * B * m1;
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_RESIDUE_ROWS, st, (double)rows * (3.0 * fft_flops((double)m2) + 14.0 * m2),
                   3.0 * rows * m2 * sizeof(V));
    kern<<<(unsigned)rows, thr, smem, st>>>(ya, yb, yh, B, (int)m1, (int)m2, (int)q, (int)r0, twm, twml, fp);
    return cudaGetLastError();
}

// Outer axis of an N-D problem, real inputs: in the mixed domain (axis 0
// transformed, inner axes not) the partner of row l0 of kept residue r is
// row l0' of r' at the same inner position (in wa itself for the
// self-paired residues r = 0 and 2 r = q, else in wb), so F and G rows are
// formed elementwise into wf and wg.  Layout [rr][b][l0][c], c < Cn.
template <class V>
__global__ void k_pair_rows_real(const V* __restrict__ wa, const V* __restrict__ wb, V* wf, V* wg, int64_t B,
                                 int64_t Cn, int m0, int q, int r0, int Dg)
{
    const int64_t per = (int64_t)m0 * Cn;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= (int64_t)Dg * B * per) return;
    const int64_t blkrow = div_idx(gid, per);
    const int64_t e = gid - blkrow * per;
    const int l0 = (int)div_idx(e, Cn);
    const int64_t c = e - (int64_t)l0 * Cn;
    const int rr = (int)(blkrow / B);
    const int r = r0 + rr;
    const int l0p = r == 0 ? (m0 - l0) % m0 : m0 - 1 - l0;
    using T = typename real_of<V>::type;
    const T h = (T)0.5;
    const V a = wa[gid];
    const V* src = (r == 0 || 2 * r == q) ? wa : wb;
    const V bb = src[blkrow * per + (int64_t)l0p * Cn + c];
    wf[gid] = mkc<V>(h * (a.x + bb.x), h * (a.y - bb.y));
    wg[gid] = mkc<V>(h * (a.y + bb.y), -h * (a.x - bb.x));
}

template <typename T>
cudaError_t launch_pair_rows_real(const cx<T>* wa, const cx<T>* wb, cx<T>* wf, cx<T>* wg, int64_t B, int64_t Cn,
                                  int64_t m0, int64_t q, int64_t r0, int64_t Dg, cudaStream_t st)
{
    const int64_t n = Dg * B * m0 * Cn;
    if (n <= 0) return cudaSuccess;
    const int thr = 256;
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_UNFOLD, st, 8.0 * n, 4.0 * n * sizeof(cx<T>));
    k_pair_rows_real<cx<T>><<<(unsigned)((n + thr - 1) / thr), thr, 0, st>>>(wa, wb, wf, wg, B, Cn, (int)m0, (int)q,
                                                                           (int)r0, (int)Dg);
    return cudaGetLastError();
}

// Unfold of kept residues into a real output: out[b][lin - lo] for
// lin = (t ma + i) Cn + c in [lo, hi) gets sum_rr w_r Re(conj(zeta_Nf^{r (i cs +
// c cc)}) conj(zeta_q^{r t}) h[rr][b][i][c]) with w_r = 1 for the
// self-paired residues (r = 0, 2 r = q) and 2 otherwise; added to the
// previous contents unless first, scaled if last.
template <class V>
__global__ void k_unfold_real(typename real_of<V>::type* out, const V* __restrict__ h, int64_t B, int64_t bstride,
                              int64_t Cn, int64_t ma, int p, int q, int64_t Nf, int64_t cs, int64_t cc, int64_t lo,
                              int64_t hi, int r0, int Dg, int first, int last, typename real_of<V>::type scale,
                              const TwTab<V> twNf)
{
    using T = typename real_of<V>::type;
    const int64_t per = ma * Cn;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= per * B) return;
    const int64_t b = div_idx(gid, per);
    const int64_t e = gid - b * per;
    const int64_t i = div_idx(e, Cn), c = e - i * Cn;
    const int64_t mq = Nf / q;
    T* ob = out + b * bstride;
    const V* hb = h + b * per;
    const int64_t hstride = B * per;
    for (int t = 0; t < p; ++t) {
        const int64_t lin = ((int64_t)t * ma + i) * Cn + c;
        if (lin >= hi) break;
        if (lin < lo) continue;
        T acc = 0;
        for (int rr = 0; rr < Dg; ++rr) {
            const int r = r0 + rr;
            const T w = (r == 0 || 2 * r == q) ? (T)1 : (T)2;
            V hv = hb[(int64_t)rr * hstride + i * Cn + c];
            if (r != 0) {
                hv = cmulc(hv, twn(twNf, (int64_t)r * (i * cs + c * cc)));
                if (t != 0) hv = cmulc(hv, twn(twNf, rt_mod(r, t, q) * mq));
            }
            acc += w * hv.x;
        }
        T v = acc;
        if (!first) v += ob[lin - lo];
        if (last) v *= scale;
        ob[lin - lo] = v;
    }
}

template <typename T>
cudaError_t launch_unfold_real(T* out, const cx<T>* h, int64_t B, int64_t bstride, int64_t Cn, int64_t ma,
                               int64_t p, int64_t q, int64_t Nf, int64_t cs, int64_t cc, int64_t lo, int64_t hi,
                               int64_t r0, int64_t Dg, int first, int last, double scale, cudaStream_t st)
{
    using V = cx<T>;
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const TwTab<V> twNf = tw_table<T>(Nf, &e);
    if (e != cudaSuccess) return e;
    const int thr = 256;
    const int64_t total = ma * Cn * B;
    const double nout = (double)(hi - lo);
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_UNFOLD, st, (double)(Dg * B) * 8.0 * nout,
                   ((double)(Dg * B * ma * Cn) * sizeof(V) + (first ? 1.0 : 2.0) * B * nout * sizeof(T)));
    k_unfold_real<V><<<(unsigned)((total + thr - 1) / thr), thr, 0, st>>>(out, h, B, bstride, Cn, ma, (int)p, (int)q,
                                                                        Nf, cs, cc, lo, hi, (int)r0, (int)Dg, first,
                                                                        last, (T)scale, twNf);
    return cudaGetLastError();
}

// ------------------------------------------------ Hermitian expansion
// full[b][x][y] (x, y in [0, 2c], c = K - 1) of the centered spectrum from
// its half half[b][x][ky] (ky in [0, c]): f(kx, ky) for ky >= 0, and
// conj(f(-kx, -ky)) for ky < 0 (the spectrum of a real field).

// ---------------------------------------- launchers with caller twiddles
// The same kernels with the twiddle tables passed in (for callers that keep
// the tables in memory of their own instead of the library cache).

template <typename T>
cudaError_t launch_twiddle_into(cx<T>* tw, int64_t n, cudaStream_t st)
{
    return launch_twiddle<T>(tw, n, st);
}

// tw[i] = zeta_N^{(i stride) mod N}, i < count, from one FP64 sincospi of the
// exact integer angle each (the two tables of a large TwTab)
template <class V>
__global__ void k_twiddle_strided(V* tw, int64_t count, int64_t N, int64_t stride)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t k = (int64_t)(((unsigned long long)i * (unsigned long long)stride) % (unsigned long long)N);
    const int64_t kk = (2 * k > N) ? k - N : k;
    double s, c;
    sincospi(2.0 * (double)kk / (double)N, &s, &c);
    using T = typename real_of<V>::type;
    tw[i] = mkc<V>((T)c, (T)s);
}

template <typename T>
cudaError_t launch_twiddle_strided(cx<T>* tw, int64_t count, int64_t N, int64_t stride, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const int thr = 256;
    LaunchScope ls(K_TWIDDLE, st, 0.0, 16.0 * count);
    k_twiddle_strided<cx<T>><<<(unsigned)((count + thr - 1) / thr), thr, 0, st>>>(tw, count, N, stride);
    return cudaGetLastError();
}

// tw[c ma + l] = zeta_{ma Cn}^{l c}, l < ma, c < Cn: the four-step twiddles
// of an ma x Cn split in the order a column tile reads them
template <class V>
__global__ void k_twiddle_colmajor(V* tw, int64_t ma, int64_t Cn)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = ma * Cn;
    if (idx >= n) return;
    const int64_t c = idx / ma, l = idx - c * ma;
    const int64_t k = (l * c) % n;
    const int64_t kk = (2 * k > n) ? k - n : k;
    double s, co;
    sincospi(2.0 * (double)kk / (double)n, &s, &co);
    using T = typename real_of<V>::type;
    tw[idx] = mkc<V>((T)co, (T)s);
}

template <typename T>
cudaError_t launch_twiddle_colmajor(cx<T>* tw, int64_t ma, int64_t Cn, cudaStream_t st)
{
    const int64_t n = ma * Cn;
    if (n <= 0) return cudaSuccess;
    const int thr = 256;
    LaunchScope ls(K_TWIDDLE, st, 0.0, 16.0 * n);
    k_twiddle_colmajor<cx<T>><<<(unsigned)((n + thr - 1) / thr), thr, 0, st>>>(tw, ma, Cn);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_twiddle_fft_into(cx<T>* tw, const FftPlan& fp, bool lf, cudaStream_t st)
{
    int64_t ns = 1;
    for (int s = 0; s < fp.nst; ++s) {
        if (ns > 1) {
            const int64_t len = ns * fp.rad[s];
            cudaError_t e = lf ? launch_twiddle_lf<T>(tw + fp.toff[s], len, st) : launch_twiddle<T>(tw + fp.toff[s], len, st);
            if (e != cudaSuccess) return e;
        }
        ns *= fp.rad[s];
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_residue_rows_tw(const cx<T>* f, const cx<T>* g, cx<T>* h, int64_t B, int64_t ld_in,
                                   int64_t L, int64_t m, int64_t p, int64_t q, int64_t r0, int64_t D,
                                   const cx<T>* twN, const cx<T>* twm, const cx<T>* twml, cudaStream_t st)
{
    using V = cx<T>;
    const int64_t Dg = (D < q - r0) ? D : (q - r0);
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const FftPlan fp = fft_plan<T>(m, rows_r16(m));
    const int thr = threads_for(m);
    const size_t smem = (size_t)(3 * smem_len<V>(m)) * sizeof(V);
    auto kern = takes_r16<V>(fp) ? k_residue_rows<V, kHas16<V>> : k_residue_rows<V, false>;
    if ((e = allow_smem(kern, smem)) != cudaSuccess) return e;
    const int64_t blocks = B * Dg;
    const double Lrow = (double)((L < p * m) ? L : p * m);
    const double fold = (p == 1 && q == 1) ? 0.0 : 16.0 * Lrow;
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_RESIDUE_ROWS, st, (double)(B * Dg) * (3.0 * fft_flops((double)m) + 6.0 * m + fold),
                   (2.0 * B * Lrow + (double)(Dg * B * m)) * sizeof(V));
    kern<<<(unsigned)blocks, thr, smem, st>>>(f, g, h, B, ld_in, ld_in, L, L, (int)m, (int)p, (int)q, (int)r0,
                                              (int)Dg, TwTab<V>{ twN, nullptr, nullptr, 0 }, twm, twml, fp);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unfold_tw(cx<T>* out, const cx<T>* h, int64_t B, int64_t bstride, int64_t Cn, int64_t ma,
                             int64_t p, int64_t q, int64_t Nf, int64_t cs, int64_t cc, int64_t Lvalid,
                             int64_t r0, int64_t D, int first, int last, double scale, const cx<T>* twNf,
                             cudaStream_t st)
{
    using V = cx<T>;
    const int64_t Dg = (D < q - r0) ? D : (q - r0);
    if (B <= 0 || Dg <= 0) return cudaSuccess;
    const int thr = 256;
    const int64_t total = ma * Cn * B;
    const int64_t blocks = (total + thr - 1) / thr;
    if (preparing()) return cudaSuccess;
    LaunchScope ls(K_UNFOLD, st, (double)(Dg * B) * 8.0 * Lvalid + (last ? 2.0 * B * Lvalid : 0.0),
                   ((double)(Dg * B * ma * Cn) + (first ? 1.0 : 2.0) * B * Lvalid) * sizeof(V));
    k_unfold<V, 4><<<(unsigned)blocks, thr, 0, st>>>(out, h, B, bstride, Cn, ma, (int)p, (int)q, Nf, cs, cc,
                                                     (int64_t)0, Lvalid, (int)r0, (int)Dg, first, last, (T)scale,
                                                     TwTab<V>{ twNf, nullptr, nullptr, 0 });
    return cudaGetLastError();
}

#define HDC_INST_TW(T)                                                                                    \
    template cudaError_t launch_twiddle_into<T>(cx<T>*, int64_t, cudaStream_t);                          \
    template cudaError_t launch_twiddle_fft_into<T>(cx<T>*, const FftPlan&, bool, cudaStream_t);          \
    template cudaError_t launch_twiddle_strided<T>(cx<T>*, int64_t, int64_t, int64_t, cudaStream_t);      \
    template cudaError_t launch_twiddle_colmajor<T>(cx<T>*, int64_t, int64_t, cudaStream_t);              \
    template cudaError_t launch_residue_rows_tw<T>(const cx<T>*, const cx<T>*, cx<T>*, int64_t, int64_t, \
                                                   int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, \
                                                   const cx<T>*, const cx<T>*, const cx<T>*, cudaStream_t); \
    template cudaError_t launch_unfold_tw<T>(cx<T>*, const cx<T>*, int64_t, int64_t, int64_t, int64_t,   \
                                             int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,       \
                                             int64_t, int64_t, int, int, double, const cx<T>*,           \
                                             cudaStream_t);

HDC_INST_TW(double)
HDC_INST_TW(float)

// ------------------------------------------------------ instantiations

#define HDC_INST_IU(T)                                                                                    \
    template cudaError_t launch_ifft_unfold<T>(cx<T>*, cx<T>*, int64_t, int64_t, int64_t, int64_t, int64_t, \
                                               int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,        \
                                               int64_t, int64_t, int, int, double, int, cudaStream_t);

HDC_INST_IU(double)
HDC_INST_IU(float)

#define HDC_INST_REAL(T)                                                                                  \
    template cudaError_t launch_pack_real<T>(const T*, const T*, cx<T>*, int64_t, cudaStream_t);        \
    template cudaError_t launch_residue_rows_real<T>(const cx<T>*, cx<T>*, int64_t, int64_t, int64_t,    \
                                                     int64_t, int64_t, int64_t, int64_t, int64_t,        \
                                                     cudaStream_t);                                      \
    template cudaError_t launch_rows_real_pair<T>(const cx<T>*, const cx<T>*, cx<T>*, int64_t, int64_t,  \
                                                  int64_t, int64_t, int64_t, int64_t, cudaStream_t);     \
    template cudaError_t launch_pair_rows_real<T>(const cx<T>*, const cx<T>*, cx<T>*, cx<T>*, int64_t,   \
                                                  int64_t, int64_t, int64_t, int64_t, int64_t,           \
                                                  cudaStream_t);                                         \
    template cudaError_t launch_unfold_real<T>(T*, const cx<T>*, int64_t, int64_t, int64_t, int64_t,     \
                                               int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,     \
                                               int64_t, int64_t, int64_t, int, int, double, cudaStream_t);

HDC_INST_REAL(double)
HDC_INST_REAL(float)

#define HDC_INST(T)                                                                                       \
    template cudaError_t launch_residue_rows<T>(const cx<T>*, const cx<T>*, cx<T>*, int64_t, int64_t,   \
                                                int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,   \
                                                int64_t, int64_t, cudaStream_t);                        \
    template cudaError_t launch_residue_rows_lam<T>(const cx<T>*, const cx<T>*, cx<T>*, int64_t, int64_t, \
                                                    int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, \
                                                    int64_t, int64_t, int64_t, int64_t, cudaStream_t);    \
    template cudaError_t launch_residue_rows_multi<T>(const cx<T>* const*, int, int, cx<T>*, int64_t,      \
                                                      int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, \
                                                      int64_t, cudaStream_t);                               \
    template cudaError_t launch_fold_fft_cols<T>(const ColSide<T>*, int, int64_t, int64_t, int64_t,     \
                                                 int64_t, int64_t, int64_t, int64_t, int64_t, int,      \
                                                 cudaStream_t);                                         \
    template cudaError_t launch_ifft_cols<T>(cx<T>*, int64_t, int64_t, int64_t, int64_t, int64_t,      \
                                             int64_t, int, cudaStream_t);                               \
    template cudaError_t launch_unfold<T>(cx<T>*, const cx<T>*, int64_t, int64_t, int64_t, int64_t,     \
                                          int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,         \
                                          int64_t, int64_t, int64_t, int, int, double, cudaStream_t);

HDC_INST(double)
HDC_INST(float)

} // namespace hdc

HDC_EXPORT int hdc_set_tma(int enable)
{
    hdc::g_fold_tma.store(enable ? 1 : 0);
    return HDC_OK;
}

HDC_EXPORT int hdc_device_status(int* status, int clear)
{
    if (!status) return HDC_ERR_PARAM;
    if (cudaDeviceSynchronize() != cudaSuccess) return HDC_ERR_CUDA;
    if (cudaMemcpyFromSymbol(status, hdc::g_device_status, sizeof(int)) != cudaSuccess) return HDC_ERR_CUDA;
    if (clear && *status != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(hdc::g_device_status, &zero, sizeof(int)) != cudaSuccess) return HDC_ERR_CUDA;
    }
    return HDC_OK;
}

// hdc_cluster.cu -- whole 1-D convolutions of short rows on a thread-block
// cluster: every residue's fold, forward transforms, product, inverse
// transform and unfold run in one launch, with the m-point transforms spread
// over the cluster's C blocks and exchanged through distributed shared
// memory, and each output written once at the end.
//
// A row's transforms on one block are bound by that SM's FP64 rate (two
// lanes per clock), so a short convolution on the one-block-per-residue
// routes takes tens of microseconds however little work it has; spread over
// C SMs the same work takes about 1/C of that, and nothing goes back to
// global memory between the steps (Section 2.2, Eq. 1 and Eq. 2: the
// residues are independent until the unfold sum, which is kept on chip).
//
// The m-point DFT of a residue is taken in four steps, m = m1 m2,
// s = s1 m2 + s2, l = l1 + m1 l2:
//   W[l1 + m1 l2] = sum_{s2} zeta_{m2}^{l2 s2} zeta_m^{l1 s2} sum_{s1} zeta_{m1}^{l1 s1} w[s1 m2 + s2].
// Block c of the cluster owns the columns s2 in [c w2, (c+1) w2) (w2 = m2/C)
// for the fold, the m1-point column transforms, the inverse column
// transforms and the unfold, and the rows l1 in [c w1, (c+1) w1)
// (w1 = m1/C) for the m2-point row transforms and the product; the
// transpose between the two layouts reads the other blocks' tiles with
// plain loads from their shared memory (no multicast).  Residues run one
// after another (r increasing, the summation order of the other routes), so
// the on-chip footprint is one residue's: the paper's D = 1.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <map>
#include <stdint.h>

#include "hdc.h"
#include "hdc_fft.cuh"
#include "hdc_internal.h"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace cg = cooperative_groups;

namespace hdc {

// The cluster route (hdc_set_cluster): 0 off, 1 where it is the faster
// route, 2 wherever the residue fits a cluster.
static std::atomic<int> g_cluster_route{ 1 };
int cluster_route_mode() { return g_cluster_route.load(); }

// x / d for x >= 0: a shift when d is a power of two (sh >= 0), else a
// division (about twenty integer instructions)
struct IDiv {
    int d, sh;
    __device__ __forceinline__ int div(int x) const { return sh >= 0 ? (x >> sh) : x / d; }
};
static IDiv make_idiv(int d)
{
    IDiv r{ d, -1 };
    if (d > 0 && (d & (d - 1)) == 0) {
        r.sh = 0;
        while ((1 << r.sh) < d) ++r.sh;
    }
    return r;
}

template <class V> struct ClusterArgs {
    const V* f;
    const V* g;
    V* out;
    int64_t ld_f, ld_g, ldo;  // row strides
    int64_t L;                // valid input elements per row
    int64_t lo, hi;           // output window [lo, hi) of each row
    int m, m1, m2, p, q, pout;
    int r_lo, r_hi;           // residues [r_lo, r_hi)
    typename real_of<V>::type scale;
    TwTab<V> twN;             // zeta_N^k, N = q m
    const V* tw1;             // stage tables of the m1-point transform
    const V* tw1l;
    const V* tw2;             // ... of the m2-point transform
    const V* tw2l;
    FftPlan fp1, fp2;
    IDiv dm1, dm2, dw1, dw2;  // m1, m2, m1 / C, m2 / C
    int stage;                // the inputs are staged in shared memory
    int lg1, lg2;             // log2 m1, log2 m2 (the shuffle transforms)
};

// Shared memory of one block (elements): the column tile X and the row tile
// Y (each holds f and g side by side: two tiles of m / C), a scratch half S
// of the same size for the transforms (no other block reads it), pout tiles
// of output accumulators, and copies of every twiddle the block reads: the
// stage tables of both transform sizes (plain and scale-tangent forms), the
// four-step twiddles of both transposes (a tile each), the residue's fold
// and unfold twiddles zeta_N^{r s} of the block's elements (a tile, made
// again for every residue) and zeta_q^k (q entries).  With the twiddles in
// shared memory, a residue waits on global memory only once, in the fold.
struct ClusterSmem {
    int tl2, tile, pout, t1, t2, q, p; // tl2: elements of a two-tile buffer
    __host__ __device__ int x() const { return 0; }
    __host__ __device__ int y() const { return tl2; }
    __host__ __device__ int scratch() const { return 2 * tl2; }
    __host__ __device__ int acc() const { return 3 * tl2; }
    __host__ __device__ int tw1() const { return acc() + pout * tile; }
    __host__ __device__ int tw1l() const { return tw1() + t1; }
    __host__ __device__ int tw2() const { return tw1l() + t1; }
    __host__ __device__ int tw2l() const { return tw2() + t2; }
    __host__ __device__ int fw() const { return tw2l() + t2; }
    __host__ __device__ int bw() const { return fw() + tile; }
    __host__ __device__ int ft() const { return bw() + tile; }
    __host__ __device__ int ft2() const { return ft() + tile; }
    __host__ __device__ int in() const { return ft2() + tile; }
    __host__ __device__ int qt() const { return in() + 2 * p * tile; } // p = 0: inputs not staged
    __host__ __device__ int total() const { return qt() + q; }
};

// Asynchronous 8- or 16-byte copy from global to shared memory (cp.async,
// completed by this thread's cp_async_wait_all).
template <class V> __device__ __forceinline__ void cp_async_el(V* smem, const V* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(V) == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// zeta_N^k into shared memory: by cp.async from a whole table, else (a
// large FP32 table kept as two) computed here
template <class V> __device__ __forceinline__ void twn_to_smem(V* dst, const TwTab<V>& t, int64_t k)
{
    if (t.full) cp_async_el(dst, t.full + k);
    else *dst = twn(t, k);
}

// n-point transforms (n = 2^lg <= 64) held in registers by groups of
// G = min(n, 32) consecutive lanes, K = n / G points per lane (lane i holds
// the points p = i + G k), with no block barrier: radix-2 stages of span
// h < G take the partner's value (point p ^ h) by a warp shuffle, and every
// lane of the warp must take part; with K = 2 the stage of span n / 2 pairs
// a lane's own two points.  twl: the packed table of the n-point radix-2
// plan in the twiddle-merged form (the stage of span h = 2^s >= 2 at offset
// 2^{s+1} - 4, entry k = zeta_{2h}^k).

// one decimation-in-time stage of span h = 2^st < G: each lane forms its own
// output a + w b (lower lane) or a - w b (upper lane) of its pair,
// w = zeta_{2h}^{p mod h}: 4 FMAs
template <class V, bool INV> __device__ __forceinline__ V dit_stage(V x, int i, int st, const V* twl)
{
    using T = typename real_of<V>::type;
    const int h = 1 << st;
    V y;
    y.x = __shfl_xor_sync(0xffffffffu, x.x, h);
    y.y = __shfl_xor_sync(0xffffffffu, x.y, h);
    const bool up = (i & h) != 0;
    const V a = up ? y : x, b = up ? x : y;
    if (st == 0) {
        const T sg = up ? (T)-1 : (T)1;
        return mkc<V>(fma(sg, b.x, a.x), fma(sg, b.y, a.y));
    }
    const LfW<V> w = lf_load<V, INV, true>(twl + ((2 << st) - 4), i & (h - 1));
    const T ux = INV ? fma(w.tt, b.y, b.x) : fma(-w.tt, b.y, b.x);
    const T uy = INV ? fma(-w.tt, b.x, b.y) : fma(w.tt, b.x, b.y);
    const T px = w.f1 ? uy : ux;
    const T py = w.f1 ? ux : uy;
    return mkc<V>(fma(flip_sign_if(w.sx, up), px, a.x), fma(flip_sign_if(w.sy, up), py, a.y));
}

// d w in the twiddle-merged form
template <class V, bool INV> __device__ __forceinline__ V lf_apply(V d, const LfW<V>& w)
{
    using T = typename real_of<V>::type;
    const T ux = INV ? fma(w.tt, d.y, d.x) : fma(-w.tt, d.y, d.x);
    const T uy = INV ? fma(-w.tt, d.x, d.y) : fma(w.tt, d.x, d.y);
    const T px = w.f1 ? uy : ux;
    const T py = w.f1 ? ux : uy;
    return mkc<V>(w.sx * px, w.sy * py);
}

// one decimation-in-frequency stage of span h = 2^st < G: the lower lane of
// a pair keeps a + b and the upper one (a - b) w, w = zeta_{2h}^{p mod h}
// (w = 1 for the lower lane, so both run the same 6 FP64 instructions)
template <class V, bool INV> __device__ __forceinline__ V dif_stage(V x, int i, int st, const V* twl)
{
    using T = typename real_of<V>::type;
    const int h = 1 << st;
    V y;
    y.x = __shfl_xor_sync(0xffffffffu, x.x, h);
    y.y = __shfl_xor_sync(0xffffffffu, x.y, h);
    const bool up = (i & h) != 0;
    const V a = up ? y : x, b = up ? x : y;
    const T sg = up ? (T)-1 : (T)1;
    const V d = mkc<V>(fma(sg, b.x, a.x), fma(sg, b.y, a.y));
    if (st == 0) return d;
    LfW<V> w;
    if (up) {
        w = lf_load<V, INV, true>(twl + ((2 << st) - 4), i & (h - 1));
    } else {
        w.sx = (T)1;
        w.sy = (T)1;
        w.tt = (T)0;
        w.f1 = false;
    }
    return lf_apply<V, INV>(d, w);
}

// Decimation in time: point p enters as x[bitrev(p)] and leaves as X[p].
template <class V, bool INV> __device__ __forceinline__ void warp_dit(V* x, int i, int lg, int K, const V* twl)
{
    const int lgG = lg - (K - 1);
    for (int st = 0; st < lgG; ++st) {
        x[0] = dit_stage<V, INV>(x[0], i, st, twl);
        if (K == 2) x[1] = dit_stage<V, INV>(x[1], i, st, twl);
    }
    // span n / 2: points i and i + n / 2, both in this lane
    if (K == 2) lf_bfly<V, INV>(x[0], x[1], lf_load<V, INV, true>(twl + ((2 << (lg - 1)) - 4), i));
}

// Decimation in frequency: point p enters as x[p] and leaves as X[bitrev(p)].
template <class V, bool INV> __device__ __forceinline__ void warp_dif(V* x, int i, int lg, int K, const V* twl)
{
    const int lgG = lg - (K - 1);
    if (K == 2) {
        const V a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = lf_apply<V, INV>(csub(a, b), lf_load<V, INV, true>(twl + ((2 << (lg - 1)) - 4), i));
    }
    for (int st = lgG - 1; st >= 0; --st) {
        x[0] = dif_stage<V, INV>(x[0], i, st, twl);
        if (K == 2) x[1] = dif_stage<V, INV>(x[1], i, st, twl);
    }
}

// KW > 0: the m1- and m2-point transforms (powers of two up to 32 points
// for KW = 1, up to 64 for KW = 2) by warp shuffles (warp_dit, warp_dif)
// instead of the shared-memory stages.
template <class V, int KW>
__global__ void __launch_bounds__(kMaxThreads) k_conv_cluster(const __grid_constant__ ClusterArgs<V> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int c = (int)cluster.block_rank();
    const int64_t b = blockIdx.x / C;
    const int w1 = a.m1 / C, w2 = a.m2 / C;
    const int tile = a.m / C;
    const ClusterSmem L{ (int)smem_len<V>(2 * tile), tile, a.pout, a.fp1.tlen, a.fp2.tlen, a.q, a.stage ? a.p : 0 };
    V* sm = reinterpret_cast<V*>(smraw);
    // X: element (s1, col) at s1 (2 w2) + col, f in columns [0, w2), g in
    // [w2, 2 w2); Y: element (s2, col) at s2 (2 w1) + col, f in [0, w1), g in
    // [w1, 2 w1)
    V* X = sm + L.x();
    V* Y = sm + L.y();
    V* S = sm + L.scratch();
    V* acc = sm + L.acc();
    V* T1 = sm + L.tw1();
    V* T1l = sm + L.tw1l();
    V* T2 = sm + L.tw2();
    V* T2l = sm + L.tw2l();
    V* FW = sm + L.fw();
    V* BW = sm + L.bw();
    V* FT = sm + L.ft();
    V* FT2 = sm + L.ft2();
    V* INF = sm + L.in();           // f at t m + s, element (t, e) at t tile + e
    V* ING = INF + a.p * tile;      // g
    V* QT = sm + L.qt();
    const int xw = 2 * w2, yw = 2 * w1;
    constexpr bool W = KW > 0;
    const int lgC = __ffs(C) - 1, lgw1 = a.lg1 - lgC, lgw2 = a.lg2 - lgC; // C, m1, m2: powers of two (W)
    const int tid = threadIdx.x, nthr = blockDim.x;
    const V* fr = a.f + b * a.ld_f;
    const V* gr = a.g + b * a.ld_g;
    // the block's copies of its twiddles (loads issued together)
    for (int e = tid; e < L.t1; e += nthr) {
        T1[e] = __ldg(a.tw1 + e);
        T1l[e] = __ldg(a.tw1l + e);
    }
    for (int e = tid; e < L.t2; e += nthr) {
        T2[e] = __ldg(a.tw2 + e);
        T2l[e] = __ldg(a.tw2l + e);
    }
    for (int e = tid; e < tile; e += nthr) {
        // forward transpose element (rl, s2): zeta_m^{l1 s2}, l1 = c w1 + rl
        const int rl = a.dm2.div(e), s2f = e - rl * a.m2;
        FW[e] = twn(a.twN, (int64_t)a.q * (c * w1 + rl) * s2f);
        // backward transpose element (cl, l1): zeta_m^{l1 s2}, s2 = c w2 + cl
        const int cl = a.dm1.div(e), l1 = e - cl * a.m1;
        BW[e] = twn(a.twN, (int64_t)a.q * l1 * (c * w2 + cl));
    }
    for (int e = tid; e < a.q; e += nthr) QT[e] = twn(a.twN, (int64_t)e * a.m);
    for (int e = tid; e < a.pout * tile; e += nthr) acc[e] = czero<V>();
    // the elements of f and g this block folds (the same for every residue;
    // staged unless the block's shared memory cannot hold them) and the
    // first residue's fold twiddles zeta_N^{r s}; later residues' twiddles
    // are copied during the residue before (cp.async), so with staged inputs
    // no residue waits on global memory
    for (int e = tid; e < tile; e += nthr) {
        const int s1 = a.dw2.div(e), cl = e - s1 * w2;
        const int64_t s = (int64_t)s1 * a.m2 + (int64_t)c * w2 + cl;
        if (a.stage)
            for (int t = 0; t < a.p; ++t) {
                const int64_t j = (int64_t)t * a.m + s;
                INF[t * tile + e] = j < a.L ? fr[j] : czero<V>();
                ING[t * tile + e] = j < a.L ? gr[j] : czero<V>();
            }
        twn_to_smem(FT + e, a.twN, (int64_t)a.r_lo * s);
    }
    cp_async_wait_all();
    __syncthreads();
    if constexpr (W) {
        // The shuffle transforms: no tile goes through shared memory between
        // the fold and the push, or between the product and the push.  In
        // the column phases the lanes of group col (G1 of them) hold the
        // m1 points of column col of the two-tile X (f in columns [0, w2),
        // g in [w2, 2 w2)), point p = i + G1 k in slot k; in the row phases
        // the G2 lanes of group col the m2 points of column col of Y.
        const int K1 = (KW == 2 && a.m1 > 32) ? 2 : 1, K2 = (KW == 2 && a.m2 > 32) ? 2 : 1;
        const int G1 = a.m1 / K1, G2 = a.m2 / K2;
        const int lgG1 = a.lg1 - (K1 - 1), lgG2 = a.lg2 - (K2 - 1);
        const int ccol = tid >> lgG1, ci = tid & (G1 - 1);
        const int cside = ccol >= w2 ? 1 : 0, ccl = ccol - cside * w2;
        const bool cact = tid < xw * G1, cwarp = (tid & ~31) < xw * G1;
        const int rcol = tid >> lgG2, ri = tid & (G2 - 1);
        const bool ract = tid < yw * G2, rwarp = (tid & ~31) < yw * G2;
        const bool iwarp = (tid & ~31) < w1 * G2;       // inverse row transforms (f rows)
        const bool uwarp = (tid & ~31) < w2 * G1;       // inverse column transforms (f columns)
        const V* in_side = cside ? ING : INF;
        const V* g_side = cside ? gr : fr;
        auto rev1 = [&](int p) { return (int)(__brev((unsigned)p) >> (32 - a.lg1)); };
        for (int r = a.r_lo; r < a.r_hi; ++r) {
            V* FTc = ((r - a.r_lo) & 1) ? FT2 : FT;
            V* FTn = ((r - a.r_lo) & 1) ? FT : FT2;
            const int rq = r % a.q;
            // fold (Eq. 1 inner sum, then zeta_N^{r s}) of element s1 =
            // bitrev(p) of this lane's column for each of its points p (the
            // order the transform reads), then the m1-point transform;
            // result l1 = p goes to the block that owns row l1, times
            // zeta_m^{l1 s2}
            if (cwarp) {
                V x[2] = { czero<V>(), czero<V>() };
                if (cact)
                    _Pragma("unroll") for (int k = 0; k < 2; ++k) if (k < K1) {
                        const int s1 = rev1(ci + G1 * k);
                        const int e = s1 * w2 + ccl;
                        const int64_t s = (int64_t)s1 * a.m2 + (int64_t)c * w2 + ccl;
                        V v = a.stage ? in_side[e] : (s < a.L ? g_side[s] : czero<V>());
                        int qi = 0;              // (r t) mod q
                        for (int t = 1; t < a.p; ++t) {
                            const int64_t j = (int64_t)t * a.m + s;
                            if (j >= a.L) break;
                            qi += rq;
                            if (qi >= a.q) qi -= a.q;
                            v = cfma(a.stage ? in_side[t * tile + e] : g_side[j], QT[qi], v);
                        }
                        x[k] = cmul(v, FTc[e]);
                    }
                warp_dit<V, false>(x, ci, a.lg1, K1, T1l);
                if (cact)
                    _Pragma("unroll") for (int k = 0; k < 2; ++k) if (k < K1) {
                        const int l1 = ci + G1 * k;
                        V* yd = cluster.map_shared_rank(Y, l1 >> lgw1);
                        yd[sidx<V, true>((c * w2 + ccl) * yw + cside * w1 + (l1 & (w1 - 1)))] =
                            cmul(x[k], BW[ccl * a.m1 + l1]);
                    }
            }
            cluster.sync();
            // the next residue's fold twiddles, copied while the rows run
            // (every read of the buffer they replace came before the barrier)
            if (r + 1 < a.r_hi)
                for (int e = tid; e < tile; e += nthr) {
                    const int s1 = a.dw2.div(e), cl = e - s1 * w2;
                    twn_to_smem(FTn + e, a.twN, (int64_t)(r + 1) * ((int64_t)s1 * a.m2 + (int64_t)c * w2 + cl));
                }
            // m2-point transforms of the rows (decimation in frequency: point
            // p ends as bin bitrev(p)); g's bins through shared memory to the
            // lane of f with the same points, product (Section 2.4), inverse
            // transform (decimation in time: point p ends as s2 = p), result
            // to the block that owns column s2, times conj(zeta_m^{l1 s2})
            V y[2] = { czero<V>(), czero<V>() };
            if (rwarp) {
                if (ract)
                    _Pragma("unroll") for (int k = 0; k < 2; ++k) if (k < K2) y[k] = Y[sidx<V, true>((ri + G2 * k) * yw + rcol)];
                warp_dif<V, false>(y, ri, a.lg2, K2, T2l);
                if (ract && rcol >= w1)
                    _Pragma("unroll") for (int k = 0; k < 2; ++k) if (k < K2) Y[sidx<V, true>((ri + G2 * k) * yw + rcol)] = y[k];
            }
            __syncthreads();
            if (iwarp) {
                const bool fact = tid < w1 * G2;
                if (fact)
                    _Pragma("unroll") for (int k = 0; k < 2; ++k) if (k < K2) y[k] = cmul(y[k], Y[sidx<V, true>((ri + G2 * k) * yw + rcol + w1)]);
                warp_dit<V, true>(y, ri, a.lg2, K2, T2l);
                if (fact)
                    _Pragma("unroll") for (int k = 0; k < 2; ++k) if (k < K2) {
                        const int s2 = ri + G2 * k;
                        V* xd = cluster.map_shared_rank(X, s2 >> lgw2);
                        xd[sidx<V, true>((c * w1 + rcol) * xw + (s2 & (w2 - 1)))] = cmulc(y[k], FW[rcol * a.m2 + s2]);
                    }
            }
            cp_async_wait_all();
            cluster.sync();
            // inverse m1-point transforms of this block's columns (point p
            // loads row bitrev(p), ends as h_r[s], s1 = p), then the unfold
            // (Eq. 2 outer sums): output j = t m + s gets
            // conj(zeta_N^{r s}) conj(zeta_q^{r t}) h_r[s]
            if (uwarp) {
                const bool uact = tid < w2 * G1;
                V x[2] = { czero<V>(), czero<V>() };
                if (uact)
                    _Pragma("unroll") for (int k = 0; k < 2; ++k) if (k < K1) x[k] = X[sidx<V, true>(rev1(ci + G1 * k) * xw + ccol)];
                warp_dit<V, true>(x, ci, a.lg1, K1, T1l);
                if (uact)
                    _Pragma("unroll") for (int k = 0; k < 2; ++k) if (k < K1) {
                        const int s1 = ci + G1 * k;
                        const int e = s1 * w2 + ccol;
                        const int64_t s = (int64_t)s1 * a.m2 + (int64_t)c * w2 + ccol;
                        const V hv = cmulc(x[k], FTc[e]);
                        int qi = 0;
                        for (int t = 0; t < a.pout; ++t) {
                            const int64_t j = (int64_t)t * a.m + s;
                            if (j >= a.hi) break;
                            if (t != 0) {
                                qi += rq;
                                if (qi >= a.q) qi -= a.q;
                            }
                            if (j < a.lo) continue;
                            const V v = t != 0 ? cmulc(hv, QT[qi]) : hv;
                            acc[t * tile + e] = cadd(acc[t * tile + e], v);
                        }
                    }
            }
            // X is next written by the other blocks after the next residue's
            // first barrier; FTc is next overwritten after that barrier too
        }
    } else {
        for (int r = a.r_lo; r < a.r_hi; ++r) {
            // this residue's twiddles (FTc) and the next one's (FTn); a thread
            // reads only the entries it copied itself
            V* FTc = ((r - a.r_lo) & 1) ? FT2 : FT;
            V* FTn = ((r - a.r_lo) & 1) ? FT : FT2;
            cp_async_wait_all();
            const int rq = r % a.q;
            // fold (Eq. 1 inner sum, then zeta_N^{r s}) of f and g into this
            // block's columns s = s1 m2 + c w2 + cl
            for (int e = tid; e < tile; e += nthr) {
                const int s1 = a.dw2.div(e), cl = e - s1 * w2;
                const int64_t s = (int64_t)s1 * a.m2 + (int64_t)c * w2 + cl;
                const V wrs = FTc[e];
                V af, ag;
                if (a.stage) {
                    af = INF[e];
                    ag = ING[e];
                } else {
                    af = s < a.L ? fr[s] : czero<V>();
                    ag = s < a.L ? gr[s] : czero<V>();
                }
                int qi = 0;                  // (r t) mod q
                for (int t = 1; t < a.p; ++t) {
                    const int64_t j = (int64_t)t * a.m + s;
                    if (j >= a.L) break;
                    qi += rq;
                    if (qi >= a.q) qi -= a.q;
                    const V w = QT[qi];
                    af = cfma(a.stage ? INF[t * tile + e] : fr[j], w, af);
                    ag = cfma(a.stage ? ING[t * tile + e] : gr[j], w, ag);
                }
                X[sidx<V, true>(s1 * xw + cl)] = cmul(af, wrs);
                X[sidx<V, true>(s1 * xw + w2 + cl)] = cmul(ag, wrs);
                if (r + 1 < a.r_hi) twn_to_smem(FTn + e, a.twN, (int64_t)(r + 1) * s);
            }
            __syncthreads();
            // m1-point transforms of the 2 w2 columns (f and g at once)
            fft_smem<V, false, true, false, true>(X, S, a.fp1, xw, xw, 1, T1, T1l, tid, nthr);
            cluster.sync();
            // transpose: rows l1 = c w1 + rl of every column s2, from the block
            // that owns s2, times zeta_m^{l1 s2}.  Four elements per thread are
            // loaded before any is stored, so the loads from the other blocks'
            // shared memory are in flight together.
            constexpr int U = 4;
            for (int e0 = tid; e0 < tile; e0 += U * nthr) {
                V v0[U], v1[U];
    #pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * nthr;
                    if (e < tile) {
                        const int rl = a.dm2.div(e), s2 = e - rl * a.m2;
                        const int src = a.dw2.div(s2), scl = s2 - src * w2;
                        const V* rx = cluster.map_shared_rank(X, src);
                        const int row = (c * w1 + rl) * xw;
                        v0[u] = rx[sidx<V, true>(row + scl)];
                        v1[u] = rx[sidx<V, true>(row + w2 + scl)];
                    }
                }
    #pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * nthr;
                    if (e < tile) {
                        const int rl = a.dm2.div(e), s2 = e - rl * a.m2;
                        const V w = FW[e];
                        Y[sidx<V, true>(s2 * yw + rl)] = cmul(v0[u], w);
                        Y[sidx<V, true>(s2 * yw + w1 + rl)] = cmul(v1[u], w);
                    }
                }
            }
            // no cluster barrier here: this block's column tiles X are next
            // written by the transpose back, after the barrier below, which every
            // block reaches only after its own forward transpose
            __syncthreads();
            // m2-point transforms of the 2 w1 rows, product (Section 2.4), inverse
            fft_smem<V, false, true, false, true>(Y, S, a.fp2, yw, yw, 1, T2, T2l, tid, nthr);
            for (int e = tid; e < tile; e += nthr) {
                const int s2 = a.dw1.div(e), rl = e - s2 * w1;
                const int kf = sidx<V, true>(s2 * yw + rl), kg = sidx<V, true>(s2 * yw + w1 + rl);
                Y[kf] = cmul(Y[kf], Y[kg]);
            }
            __syncthreads();
            fft_smem<V, true, true, false, true>(Y, S, a.fp2, w1, yw, 1, T2, T2l, tid, nthr);
            cluster.sync();
            // transpose back: this block's columns s2 = c w2 + cl of every row l1,
            // times conj(zeta_m^{l1 s2}).  The next residue's writes to Y come
            // after its first cluster barrier, which every block reaches only
            // after this loop.
            for (int e0 = tid; e0 < tile; e0 += U * nthr) {
                V v[U];
    #pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * nthr;
                    if (e < tile) {
                        const int cl = a.dm1.div(e), l1 = e - cl * a.m1;
                        const int src = a.dw1.div(l1), rl = l1 - src * w1;
                        v[u] = cluster.map_shared_rank(Y, src)[sidx<V, true>((c * w2 + cl) * yw + rl)];
                    }
                }
    #pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * nthr;
                    if (e < tile) {
                        const int cl = a.dm1.div(e), l1 = e - cl * a.m1;
                        X[sidx<V, true>(l1 * xw + cl)] = cmulc(v[u], BW[e]);
                    }
                }
            }
            __syncthreads();
            // inverse m1-point transforms: h_r[s1 m2 + s2] of this block's columns
            fft_smem<V, true, true, false, true>(X, S, a.fp1, w2, xw, 1, T1, T1l, tid, nthr);
            // unfold (Eq. 2 outer sums): output j = t m + s gets
            // conj(zeta_N^{r s}) conj(zeta_q^{r t}) h_r[s], residues in increasing r
            for (int e = tid; e < tile; e += nthr) {
                const int s1 = a.dw2.div(e), cl = e - s1 * w2;
                const int64_t s = (int64_t)s1 * a.m2 + (int64_t)c * w2 + cl;
                const V hv = cmulc(X[sidx<V, true>(s1 * xw + cl)], FTc[e]);
                int qi = 0;                  // (r t) mod q
                for (int t = 0; t < a.pout; ++t) {
                    const int64_t j = (int64_t)t * a.m + s;
                    if (j >= a.hi) break;
                    if (t != 0) {
                        qi += rq;
                        if (qi >= a.q) qi -= a.q;
                    }
                    if (j < a.lo) continue;
                    const V v = t != 0 ? cmulc(hv, QT[qi]) : hv;
                    acc[t * tile + e] = cadd(acc[t * tile + e], v);
                }
            }
            // the thread that reads X and FTc[e] of element e here writes them in
            // the next fold, and acc entries are per thread: no barrier needed
        }
    }
    // no block leaves while another may still read its shared memory
    cluster.sync();
    for (int t = 0; t < a.pout; ++t)
        for (int e = tid; e < tile; e += nthr) {
            const int s1 = a.dw2.div(e), cl = e - s1 * w2;
            const int64_t j = (int64_t)t * a.m + (int64_t)s1 * a.m2 + (int64_t)c * w2 + cl;
            if (j >= a.lo && j < a.hi) a.out[b * a.ldo + (j - a.lo)] = cscale(acc[t * tile + e], a.scale);
        }
}

// ------------------------------------------------------------------ host

// Lanes the shuffle transforms of an m1 x m2 residue on C blocks need: the
// larger of the column phases (2 m2 / C columns of min(m1, 32) lanes) and
// the row phases (2 m1 / C columns of min(m2, 32) lanes).
static int64_t cluster_warp_lanes(int C, int64_t m1, int64_t m2)
{
    const int64_t c = 2 * (m2 / C) * (m1 < 32 ? m1 : 32), r = 2 * (m1 / C) * (m2 < 32 ? m2 : 32);
    return c > r ? c : r;
}

// Whether the cluster kernel takes the shuffle transforms for this shape:
// m1 and m2 powers of two up to 64 (at most two points per lane) and at
// most kMaxThreads lanes.
static bool cluster_warp_ffts(int64_t m, int C, int64_t m1, int64_t m2)
{
    auto pow2 = [](int64_t x) { return x > 0 && (x & (x - 1)) == 0; };
    (void)m;
    return pow2(m1) && pow2(m2) && m1 <= 64 && m2 <= 64 && cluster_warp_lanes(C, m1, m2) <= kMaxThreads;
}

// The transform plans of the cluster kernel: radix 2 throughout with the
// shuffle transforms (whose twiddles are the radix-2 stage tables), else
// the latency plans.
template <typename T> static FftPlan cluster_plan(int64_t n, bool warp_ffts)
{
    return warp_ffts ? make_fft_plan(n, false, true) : fft_plan_latency<T>(n);
}

// The kernel variant: 0 shared-memory transforms, 1 shuffle transforms of
// at most 32 points (one point per lane), 2 of up to 64 (two per lane).
static int cluster_kw(bool warp_ffts, int64_t m1, int64_t m2)
{
    return !warp_ffts ? 0 : ((m1 > 32 || m2 > 32) ? 2 : 1);
}

// Bytes of dynamic shared memory of one block (ClusterSmem).
template <typename T>
static size_t cluster_smem(int64_t m, int C, int64_t m1, int64_t m2, int64_t pout, int64_t q, int64_t p)
{
    const int64_t tile = m / C;
    const bool wf = cluster_warp_ffts(m, C, m1, m2);
    const ClusterSmem L{ (int)smem_len<cx<T>>(2 * tile), (int)tile, (int)pout, cluster_plan<T>(m1, wf).tlen,
                         cluster_plan<T>(m2, wf).tlen, (int)q, (int)p };
    return (size_t)L.total() * sizeof(cx<T>);
}

// Whether a 16-block cluster of this kernel with `smem` bytes per block can
// be resident (a non-portable size; remembered per device).
template <class V, int KW> static bool cluster16_ok(size_t smem, int thr)
{
    static std::mutex mu;
    static std::map<std::pair<int, size_t>, bool> known;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, (smem * 1024 + (size_t)thr) * 4 + (size_t)KW);
    auto it = known.find(key);
    if (it != known.end()) return it->second;
    bool ok = cudaFuncSetAttribute(k_conv_cluster<V, KW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
              cudaSuccess;
    if (ok && smem > 48 * 1024)
        ok = cudaFuncSetAttribute(k_conv_cluster<V, KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
             cudaSuccess;
    if (ok) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(thr);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        ok = cudaOccupancyMaxActiveClusters(&n, k_conv_cluster<V, KW>, &cfg) == cudaSuccess && n > 0;
    }
    cudaGetLastError();
    known[key] = ok;
    return ok;
}

// Threads of one block: one per butterfly of a stage over both inputs'
// tiles (radix 2 in FP64, radix 8 in FP32; fft_plan_latency), 64..256; with
// the shuffle transforms the lanes they need (cluster_warp_lanes).
template <typename T> static int cluster_threads(int64_t m, int C, int64_t m1, int64_t m2, bool warp_ffts)
{
    const int64_t tile = m / C;
    int thr = (int)(((warp_ffts ? cluster_warp_lanes(C, m1, m2) : (sizeof(T) == 8 ? tile : tile / 4)) + 31) / 32 * 32);
    return thr < 64 ? 64 : (thr > kMaxThreads ? kMaxThreads : thr);
}

// The cluster's shape for an m-point residue with pout output blocks and q
// residues: C in {16, 8, 4, 2} (the largest that divides both factors and
// leaves tiles of at least 32 elements; 16, a non-portable cluster size,
// only where the device can hold such a cluster), m = m1 m2 with C | m1,
// C | m2 and m1 <= m2 as close to sqrt(m) as allowed, shared memory within
// the per-block limit.  False when none exists.
template <typename T>
bool cluster_shape(int64_t m, int64_t pout, int64_t q, int64_t p, int* Co, int64_t* m1o, int64_t* m2o, bool* stage,
                   bool* warp)
{
    constexpr size_t kMaxSmem = 200 * 1024;
    for (int C : { 16, 8, 4, 2 }) {
        if (m % ((int64_t)C * C) != 0 || m / C < 32) continue;
        int64_t best = -1;
        for (int64_t m1 = C; m1 * m1 <= m; m1 += C)
            if (m % m1 == 0 && (m / m1) % C == 0) best = m1;
        if (best < 0) continue;
        // the inputs staged in shared memory where they fit
        bool stg = true;
        size_t smem = cluster_smem<T>(m, C, best, m / best, pout, q, p);
        if (smem > kMaxSmem) {
            stg = false;
            smem = cluster_smem<T>(m, C, best, m / best, pout, q, 0);
        }
        if (smem > kMaxSmem) continue;
        const bool wf = cluster_warp_ffts(m, C, best, m / best);
        const int thr16 = cluster_threads<T>(m, C, best, m / best, wf);
        const int kw = cluster_kw(wf, best, m / best);
        if (C == 16 && !(kw == 2 ? cluster16_ok<cx<T>, 2>(smem, thr16)
                                 : (kw == 1 ? cluster16_ok<cx<T>, 1>(smem, thr16)
                                            : cluster16_ok<cx<T>, 0>(smem, thr16))))
            continue;
        *Co = C;
        *m1o = best;
        *m2o = m / best;
        if (stage) *stage = stg;
        if (warp) *warp = wf;
        return true;
    }
    return false;
}
template bool cluster_shape<double>(int64_t, int64_t, int64_t, int64_t, int*, int64_t*, int64_t*, bool*, bool*);
template bool cluster_shape<float>(int64_t, int64_t, int64_t, int64_t, int*, int64_t*, int64_t*, bool*, bool*);

template <typename T>
cudaError_t launch_conv_cluster(const cx<T>* f, const cx<T>* g, cx<T>* out, int64_t B, int64_t ld_f, int64_t ld_g,
                                int64_t ldo, int64_t L, int64_t lo, int64_t hi, int64_t m, int64_t p, int64_t q,
                                int64_t r_lo, int64_t r_hi, double scale, cudaStream_t st)
{
    using V = cx<T>;
    if (B <= 0 || r_hi <= r_lo) return cudaSuccess;
    const int64_t pout = (hi + m - 1) / m;
    int C = 0;
    int64_t m1 = 0, m2 = 0;
    bool stage = false;
    if (!cluster_shape<T>(m, pout, q, p, &C, &m1, &m2, &stage)) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    ClusterArgs<V> a;
    a.twN = tw_table<T>(q * m, &e);
    if (e != cudaSuccess) return e;
    const bool wf = cluster_warp_ffts(m, C, m1, m2);
    a.fp1 = cluster_plan<T>(m1, wf);
    a.fp2 = cluster_plan<T>(m2, wf);
    a.tw1 = twiddles_fft_plan<T>(a.fp1, false, &e);
    if (e != cudaSuccess) return e;
    a.tw1l = twiddles_fft_plan<T>(a.fp1, true, &e);
    if (e != cudaSuccess) return e;
    a.tw2 = twiddles_fft_plan<T>(a.fp2, false, &e);
    if (e != cudaSuccess) return e;
    a.tw2l = twiddles_fft_plan<T>(a.fp2, true, &e);
    if (e != cudaSuccess) return e;
    a.f = f;
    a.g = g;
    a.out = out;
    a.ld_f = ld_f;
    a.ld_g = ld_g;
    a.ldo = ldo;
    a.L = L;
    a.lo = lo;
    a.hi = hi;
    a.m = (int)m;
    a.m1 = (int)m1;
    a.m2 = (int)m2;
    a.p = (int)p;
    a.q = (int)q;
    a.pout = (int)pout;
    a.r_lo = (int)r_lo;
    a.r_hi = (int)r_hi;
    a.scale = (T)scale;
    a.dm1 = make_idiv((int)m1);
    a.dm2 = make_idiv((int)m2);
    a.dw1 = make_idiv((int)(m1 / C));
    a.dw2 = make_idiv((int)(m2 / C));
    a.stage = stage ? 1 : 0;
    a.lg1 = 0;
    while ((int64_t(1) << a.lg1) < m1) ++a.lg1;
    a.lg2 = 0;
    while ((int64_t(1) << a.lg2) < m2) ++a.lg2;
    const int thr = cluster_threads<T>(m, C, m1, m2, wf);
    const int kw = cluster_kw(wf, m1, m2);
    auto kern = kw == 2 ? k_conv_cluster<V, 2> : (kw == 1 ? k_conv_cluster<V, 1> : k_conv_cluster<V, 0>);
    const size_t smem_c = cluster_smem<T>(m, C, m1, m2, pout, q, stage ? p : 0);
    if (smem_c > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c)) !=
            cudaSuccess)
        return e;
    if (preparing()) return cudaSuccess;
    // model: per row and residue 3 m-point FFTs, the product, the folds of f
    // and g and the unfold (8 flops per element each), the final scaling
    const double Lrow = (double)(L < p * m ? L : p * m);
    LaunchScope ls(K_CLUSTER, st,
                   (double)B * (r_hi - r_lo) * (3.0 * fft_flops((double)m) + 6.0 * m + 16.0 * Lrow + 8.0 * (hi - lo)) +
                       2.0 * B * (hi - lo),
                   (double)B * (2.0 * Lrow + (double)(hi - lo)) * sizeof(V));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(B * C));
    cfg.blockDim = dim3(thr);
    cfg.dynamicSmemBytes = smem_c;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
template cudaError_t launch_conv_cluster<double>(const cx<double>*, const cx<double>*, cx<double>*, int64_t, int64_t,
                                                 int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,
                                                 int64_t, int64_t, int64_t, double, cudaStream_t);
template cudaError_t launch_conv_cluster<float>(const cx<float>*, const cx<float>*, cx<float>*, int64_t, int64_t,
                                                int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,
                                                int64_t, int64_t, int64_t, double, cudaStream_t);

} // namespace hdc

HDC_EXPORT int hdc_set_cluster(int mode)
{
    if (mode < 0 || mode > 2) return HDC_ERR_PARAM;
    hdc::g_cluster_route.store(mode);
    return HDC_OK;
}

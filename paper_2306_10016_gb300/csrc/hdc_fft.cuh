// hdc_fft.cuh -- device primitives: complex arithmetic, radix-R DFT kernels
// and an in-place mixed-radix Stockham FFT staged in shared memory.
//
// Sign convention (Eq. 1 and Eq. 2): zeta_n = exp(2 pi i / n); the forward
// transform sums zeta^{+kj}, the inverse zeta^{-kj}; neither is scaled.
//
// The FFT works on `ncol` transforms at once whose element i of column c sits
// at buf[i * ld + c * cs] (ld = ncol, cs = 1 for a tile of interleaved columns,
// ld = 1, cs = n for columns stored one after another).  Each stage of radix
// R reads the R inputs of a butterfly from one shared buffer and writes its R
// outputs to their autosorted (Stockham) positions in the other:
//   inputs  j + r n/R                         (r = 0..R-1, j = 0..n/R-1)
//   twiddle zeta_{Ns R}^{r (j mod Ns)}        (Ns = product of earlier radices)
//   outputs (j div Ns) Ns R + (j mod Ns) + r Ns
// after which the data of the next stage is in order, so no bit reversal is
// ever needed.  Twiddles come from per-stage tables of zeta_{Ns R}^e (see
// FftPlan) made in FP64 from exact integer angles; radix-2, 4 and 8 stages
// after the first merge them into their butterflies from a second set of
// the same values in scale-tangent form (see lf_bfly).  FP32 plans may start
// with radix-16 stages (Dft<V, 16>), whose twiddles are products of four
// table entries.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hdc {

template <typename T> struct cvec;
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<float> { using type = float2; };
template <typename T> using cx = typename cvec<T>::type;

template <class V> struct real_of;
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<float2> { using type = float; };

template <class V> __device__ __forceinline__ V mkc(typename real_of<V>::type a, typename real_of<V>::type b)
{
    V r;
    r.x = a;
    r.y = b;
    return r;
}
template <class V> __device__ __forceinline__ V czero() { return mkc<V>(0, 0); }
template <class V> __device__ __forceinline__ V cadd(V a, V b) { return mkc<V>(a.x + b.x, a.y + b.y); }
template <class V> __device__ __forceinline__ V csub(V a, V b) { return mkc<V>(a.x - b.x, a.y - b.y); }
template <class V> __device__ __forceinline__ V cscale(V a, typename real_of<V>::type s) { return mkc<V>(a.x * s, a.y * s); }
// The complex products in explicit FMAs: the same rounding wherever the
// compiler inlines them (left to contraction, two kernels that share a body
// could round the same product differently).
// a * w
template <class V> __device__ __forceinline__ V cmul(V a, V w)
{
    return mkc<V>(fma(a.x, w.x, -(a.y * w.y)), fma(a.x, w.y, a.y * w.x));
}
// a * conj(w)
template <class V> __device__ __forceinline__ V cmulc(V a, V w)
{
    return mkc<V>(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -(a.x * w.y)));
}
// acc + a * w
template <class V> __device__ __forceinline__ V cfma(V a, V w, V acc)
{
    return mkc<V>(fma(a.x, w.x, fma(-a.y, w.y, acc.x)), fma(a.x, w.y, fma(a.y, w.x, acc.y)));
}
// acc + a * conj(w)
template <class V> __device__ __forceinline__ V cfmac(V a, V w, V acc)
{
    return mkc<V>(fma(a.x, w.x, fma(a.y, w.y, acc.x)), fma(a.y, w.x, fma(-a.x, w.y, acc.y)));
}
// multiply by +i (forward) or -i (inverse)
template <class V, bool INV> __device__ __forceinline__ V rot90(V a)
{
    return INV ? mkc<V>(a.y, -a.x) : mkc<V>(-a.y, a.x);
}

template <class V> __device__ __forceinline__ V ldg_c(const V* p) { return __ldg(p); }
// A twiddle-table entry: through the read-only cache from global memory, or
// (TS) a plain load from a copy the kernel keeps in shared memory.
template <class V, bool TS> __device__ __forceinline__ V ld_tw(const V* p)
{
    if constexpr (TS) return *p;
    else return __ldg(p);
}

// ------------------------------------------------------------ radix DFTs
// v[k] <- sum_j zeta_R^{+-jk} v[j], in registers.

template <class V, bool INV> __device__ __forceinline__ void dft2(V& a, V& b)
{
    V t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <class V, bool INV> __device__ __forceinline__ void dft4(V& x0, V& x1, V& x2, V& x3)
{
    V t0 = cadd(x0, x2), t1 = csub(x0, x2);
    V t2 = cadd(x1, x3), t3 = rot90<V, INV>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

template <class V, int R, bool INV> struct Dft;

template <class V, bool INV> struct Dft<V, 2, INV> {
    static __device__ __forceinline__ void run(V* v) { dft2<V, INV>(v[0], v[1]); }
};

template <class V, bool INV> struct Dft<V, 4, INV> {
    static __device__ __forceinline__ void run(V* v) { dft4<V, INV>(v[0], v[1], v[2], v[3]); }
};

template <class V, bool INV> struct Dft<V, 8, INV> {
    static __device__ __forceinline__ void run(V* v)
    {
        using T = typename real_of<V>::type;
        const T h = (T)0.70710678118654752440;
        V e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        V o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4<V, INV>(e0, e1, e2, e3);
        dft4<V, INV>(o0, o1, o2, o3);
        // e_k +- zeta_8^{+-k} o_k for k = 1, 3 as e +- h d with the sums and
        // differences d of o's parts: one add and two FMAs per component
        T d1x, d1y, d3x, d3y;
        if (!INV) {
            d1x = o1.x - o1.y; d1y = o1.x + o1.y;
            d3x = -(o3.x + o3.y); d3y = o3.x - o3.y;
        } else {
            d1x = o1.x + o1.y; d1y = o1.y - o1.x;
            d3x = o3.y - o3.x; d3y = -(o3.x + o3.y);
        }
        V w2 = rot90<V, INV>(o2);
        v[0] = cadd(e0, o0);
        v[4] = csub(e0, o0);
        v[1] = mkc<V>(fma(h, d1x, e1.x), fma(h, d1y, e1.y));
        v[5] = mkc<V>(fma(-h, d1x, e1.x), fma(-h, d1y, e1.y));
        v[2] = cadd(e2, w2);
        v[6] = csub(e2, w2);
        v[3] = mkc<V>(fma(h, d3x, e3.x), fma(h, d3y, e3.y));
        v[7] = mkc<V>(fma(-h, d3x, e3.x), fma(-h, d3y, e3.y));
    }
};

// 16 points as 4 x 4: with n = 4 n1 + n2 and k = k1 + 4 k2, 4-point DFTs over
// n1 for each n2, the products by zeta_16^{n2 k1} (conjugated for the
// inverse), then 4-point DFTs over n2 for each k1.  Used by the FP32
// transforms, whose stages are bound by shared-memory passes rather than
// arithmetic: 4096 points take three stages instead of four.
template <class V, bool INV> struct Dft<V, 16, INV> {
    static __device__ __forceinline__ V wmul(V a, typename real_of<V>::type c, typename real_of<V>::type s)
    {
        // a * (c + i s) forward, a * (c - i s) inverse
        return INV ? mkc<V>(a.x * c + a.y * s, a.y * c - a.x * s) : mkc<V>(a.x * c - a.y * s, a.y * c + a.x * s);
    }
    static __device__ __forceinline__ void run(V* v)
    {
        using T = typename real_of<V>::type;
        const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173; // zeta_16
        const T h = (T)0.70710678118654752440;                                   // zeta_8
        V a0[4] = { v[0], v[4], v[8], v[12] }, a1[4] = { v[1], v[5], v[9], v[13] };
        V a2[4] = { v[2], v[6], v[10], v[14] }, a3[4] = { v[3], v[7], v[11], v[15] };
        dft4<V, INV>(a0[0], a0[1], a0[2], a0[3]);
        dft4<V, INV>(a1[0], a1[1], a1[2], a1[3]);
        dft4<V, INV>(a2[0], a2[1], a2[2], a2[3]);
        dft4<V, INV>(a3[0], a3[1], a3[2], a3[3]);
        // zeta_16^{n2 k1}: n2 = 1: k1 = 1, 2, 3; n2 = 2: 2, 4, 6; n2 = 3: 3, 6, 9
        a1[1] = wmul(a1[1], c1, s1);
        a1[2] = wmul(a1[2], h, h);
        a1[3] = wmul(a1[3], s1, c1);
        a2[1] = wmul(a2[1], h, h);
        a2[2] = rot90<V, INV>(a2[2]);
        a2[3] = wmul(a2[3], -h, h);
        a3[1] = wmul(a3[1], s1, c1);
        a3[2] = wmul(a3[2], -h, h);
        a3[3] = wmul(a3[3], -c1, -s1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            V x0 = a0[k1], x1 = a1[k1], x2 = a2[k1], x3 = a3[k1];
            dft4<V, INV>(x0, x1, x2, x3);
            v[k1] = x0;
            v[k1 + 4] = x1;
            v[k1 + 8] = x2;
            v[k1 + 12] = x3;
        }
    }
};

// Odd radix R = 2H+1: X_k = x0 + sum_j cos(2 pi jk/R)(x_j + x_{R-j})
//                            +- i sum_j sin(2 pi jk/R)(x_j - x_{R-j}),
// X_{R-k} the same with the sine part negated.
template <int R> struct OddConsts;
template <> struct OddConsts<3> {
    static __device__ __forceinline__ double c(int e) { return -0.5; }
    static __device__ __forceinline__ double s(int e) { return 0.86602540378443864676; }
};
template <> struct OddConsts<5> {
    static __device__ __forceinline__ double c(int e) { return e == 1 ? 0.30901699437494742410 : -0.80901699437494742410; }
    static __device__ __forceinline__ double s(int e) { return e == 1 ? 0.95105651629515357212 : 0.58778525229247312917; }
};
template <> struct OddConsts<7> {
    static __device__ __forceinline__ double c(int e)
    {
        return e == 1 ? 0.62348980185873353053 : (e == 2 ? -0.22252093395631440429 : -0.90096886790241912624);
    }
    static __device__ __forceinline__ double s(int e)
    {
        return e == 1 ? 0.78183148246802980871 : (e == 2 ? 0.97492791218182360702 : 0.43388373911755812048);
    }
};

template <class V, int R, bool INV> struct DftOdd {
    static __device__ __forceinline__ void run(V* v)
    {
        using T = typename real_of<V>::type;
        constexpr int H = (R - 1) / 2;
        V sp[H], sm[H];
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            sp[j - 1] = cadd(v[j], v[R - j]);
            sm[j - 1] = csub(v[j], v[R - j]);
        }
        V x0 = v[0];
        V X0 = x0;
#pragma unroll
        for (int j = 0; j < H; ++j) X0 = cadd(X0, sp[j]);
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            V a = x0, b = czero<V>();
#pragma unroll
            for (int j = 1; j <= H; ++j) {
                int e = (j * k) % R;
                T sg = (T)1;
                if (e > H) { e = R - e; sg = (T)-1; }
                T cc = (T)OddConsts<R>::c(e);
                T ss = sg * (T)OddConsts<R>::s(e);
                a = mkc<V>(a.x + cc * sp[j - 1].x, a.y + cc * sp[j - 1].y);
                b = mkc<V>(b.x + ss * sm[j - 1].x, b.y + ss * sm[j - 1].y);
            }
            V ib = rot90<V, INV>(b);
            v[k] = cadd(a, ib);
            v[R - k] = csub(a, ib);
        }
        v[0] = X0;
    }
};
template <class V, bool INV> struct Dft<V, 3, INV> : DftOdd<V, 3, INV> {};
template <class V, bool INV> struct Dft<V, 5, INV> : DftOdd<V, 5, INV> {};
template <class V, bool INV> struct Dft<V, 7, INV> : DftOdd<V, 7, INV> {};

// ------------------------------------------- twiddle-merged butterflies
// A twiddled butterfly a +- w b in 6 FMAs (the tangent form of Linzer and
// Feig): the table keeps w as sc (1 + i t) with |t| <= 1 ("form 0",
// sc = cos) or as i sc (1 + i t) ("form 1", sc = sin); the form is the last
// mantissa bit of sc.  u = (1 + i t) b takes 2 FMAs; in form 1, i u swaps
// the parts and negates one, and that sign goes into the per-twiddle scale
// pair (sx, sy), so a +- w b = (a.x +- sx px, a.y +- sy py) with (px, py) =
// (u.x, u.y) or (u.y, u.x) picked by register selects: 4 more FMAs.  The
// inverse transform uses conj(w): t -> -t, and the sign of form 1 moves to
// sy.  The sign flips are integer XORs on the high word, made once per
// twiddle, so the FP64 pipe sees the 6 FMAs only.

__device__ __forceinline__ double flip_sign_if(double x, bool c)
{
    unsigned hi = (unsigned)__double2hiint(x), out;
    asm("xor.b32 %0, %1, %2;" : "=r"(out) : "r"(hi), "r"((unsigned)c << 31));
    return __hiloint2double((int)out, __double2loint(x));
}
__device__ __forceinline__ float flip_sign_if(float x, bool c)
{
    unsigned out;
    asm("xor.b32 %0, %1, %2;" : "=r"(out) : "r"(__float_as_uint(x)), "r"((unsigned)c << 31));
    return __uint_as_float(out);
}

template <class V> __device__ __forceinline__ bool lf_form(V e);
template <> __device__ __forceinline__ bool lf_form<double2>(double2 e)
{
    return (__double2loint(e.x) & 1) != 0;
}
template <> __device__ __forceinline__ bool lf_form<float2>(float2 e) { return (__float_as_int(e.x) & 1) != 0; }

template <class V> struct LfW {
    using T = typename real_of<V>::type;
    T sx, sy, tt;
    bool f1;
};

template <class V, bool INV> __device__ __forceinline__ LfW<V> lf_prep(V e)
{
    LfW<V> w;
    w.f1 = lf_form(e);
    w.tt = e.y;
    w.sx = INV ? e.x : flip_sign_if(e.x, w.f1);
    w.sy = INV ? flip_sign_if(e.x, w.f1) : e.x;
    return w;
}

template <class V, bool INV> __device__ __forceinline__ void lf_bfly(V& a, V& b, const LfW<V>& w)
{
    using T = typename real_of<V>::type;
    const T ux = INV ? fma(w.tt, b.y, b.x) : fma(-w.tt, b.y, b.x);
    const T uy = INV ? fma(-w.tt, b.x, b.y) : fma(w.tt, b.x, b.y);
    const T px = w.f1 ? uy : ux;
    const T py = w.f1 ? ux : uy;
    const V a0 = a;
    a = mkc<V>(fma(w.sx, px, a0.x), fma(w.sy, py, a0.y));
    b = mkc<V>(fma(-w.sx, px, a0.x), fma(-w.sy, py, a0.y));
}

template <class V, bool INV, bool TS = false> __device__ __forceinline__ LfW<V> lf_load(const V* __restrict__ twl, int i)
{
    return lf_prep<V, INV>(ld_tw<V, TS>(twl + i));
}

// DFT_R of (W^r x_r), W = zeta_n^k (k < n/R), as R/2 log2 R twiddle-merged
// butterflies; twl[e] = zeta_n^e in the form above.  Outputs in natural order.
template <class V, int R, bool INV, bool TS = false> struct DftLF;

template <class V, bool INV, bool TS> struct DftLF<V, 2, INV, TS> {
    static __device__ __forceinline__ void run(V* v, const V* __restrict__ twl, int k, int n)
    {
        lf_bfly<V, INV>(v[0], v[1], lf_load<V, INV, TS>(twl, k));
    }
};

template <class V, bool INV, bool TS> struct DftLF<V, 4, INV, TS> {
    // B_r = x_r +- W^2 x_{r+2}; X_0, X_2 = B_0+ +- W B_1+; X_1, X_3 = B_0- +- (i W) B_1-
    static __device__ __forceinline__ void run(V* v, const V* __restrict__ twl, int k, int n)
    {
        const LfW<V> w2 = lf_load<V, INV, TS>(twl, 2 * k), w1 = lf_load<V, INV, TS>(twl, k),
                     wi = lf_load<V, INV, TS>(twl, k + n / 4);
        lf_bfly<V, INV>(v[0], v[2], w2);
        lf_bfly<V, INV>(v[1], v[3], w2);
        lf_bfly<V, INV>(v[0], v[1], w1);  // v0 = X0, v1 = X2
        lf_bfly<V, INV>(v[2], v[3], wi);  // v2 = X1, v3 = X3
        const V x1 = v[2], x2 = v[1];
        v[1] = x1;
        v[2] = x2;
    }
};

template <class V, bool INV, bool TS> struct DftLF<V, 8, INV, TS> {
    // B_r = x_r +- W^4 x_{r+4}; evens: E_r = B_r+ +- W^2 B_{r+2}+, X_0/4 = E_0+ +- W E_1+,
    // X_2/6 = E_0- +- (iW) E_1-; odds (V = zeta_8 W): F_r = B_r- +- (i W^2) B_{r+2}-,
    // X_1/5 = F_0+ +- (zeta_8 W) F_1+, X_3/7 = F_0- +- (zeta_8^3 W) F_1-
    static __device__ __forceinline__ void run(V* v, const V* __restrict__ twl, int k, int n)
    {
        const int e8 = n / 8;
        const LfW<V> w4 = lf_load<V, INV, TS>(twl, 4 * k);
        lf_bfly<V, INV>(v[0], v[4], w4);
        lf_bfly<V, INV>(v[1], v[5], w4);
        lf_bfly<V, INV>(v[2], v[6], w4);
        lf_bfly<V, INV>(v[3], v[7], w4);
        // v0..3 = B+, v4..7 = B-
        const LfW<V> w2 = lf_load<V, INV, TS>(twl, 2 * k), w2i = lf_load<V, INV, TS>(twl, 2 * k + 2 * e8);
        lf_bfly<V, INV>(v[0], v[2], w2);   // E0+, E0-
        lf_bfly<V, INV>(v[1], v[3], w2);   // E1+, E1-
        lf_bfly<V, INV>(v[4], v[6], w2i);  // F0+, F0-
        lf_bfly<V, INV>(v[5], v[7], w2i);  // F1+, F1-
        const LfW<V> w1 = lf_load<V, INV, TS>(twl, k), wi = lf_load<V, INV, TS>(twl, k + 2 * e8);
        const LfW<V> z1 = lf_load<V, INV, TS>(twl, k + e8), z3 = lf_load<V, INV, TS>(twl, k + 3 * e8);
        lf_bfly<V, INV>(v[0], v[1], w1);   // X0, X4
        lf_bfly<V, INV>(v[2], v[3], wi);   // X2, X6
        lf_bfly<V, INV>(v[4], v[5], z1);   // X1, X5
        lf_bfly<V, INV>(v[6], v[7], z3);   // X3, X7
        const V X0 = v[0], X4 = v[1], X2 = v[2], X6 = v[3], X1 = v[4], X5 = v[5], X3 = v[6], X7 = v[7];
        v[0] = X0; v[1] = X1; v[2] = X2; v[3] = X3;
        v[4] = X4; v[5] = X5; v[6] = X6; v[7] = X7;
    }
};

// ------------------------------------------------ zeta_N^k of a fold/unfold
// The fold and unfold twiddles zeta_N^k, k < N = q m, come from one table of
// N entries (`full`) while it is small, and always in FP64; a large FP32 one
// is replaced by two tables,
// zeta_N^k = hi[k >> lb] lo[k & (2^lb - 1)] with hi[j] = zeta_N^{j 2^lb} and
// lo[j] = zeta_N^j, each entry one exact-angle FP64 sincospi rounded once:
// one more rounding and a complex product per twiddle instead of a gather
// from a table of up to 2^25 entries, whose misses went to DRAM.
template <class V> struct TwTab {
    const V* full; // N entries, or null
    const V* hi;   // ceil(N / 2^lb) entries
    const V* lo;   // 2^lb entries
    int lb;
};

template <class V> __device__ __forceinline__ V twn(const TwTab<V>& t, int64_t k)
{
    if constexpr (sizeof(V) == 16) {
        return __ldg(t.full + k); // FP64 keeps whole tables (see tw_table)
    } else {
        if (t.full) return __ldg(t.full + k);
        // the product in explicit FMAs, so it rounds the same wherever the
        // compiler inlines it
        const V h = __ldg(t.hi + (k >> t.lb)), l = __ldg(t.lo + (k & (((int64_t)1 << t.lb) - 1)));
        return mkc<V>(fma(h.x, l.x, -(h.y * l.y)), fma(h.x, l.y, h.y * l.x));
    }
}

// ---------------------------------------------------------- FFT plan

#define HDC_MAX_STAGES 32

// Most inputs of one multi-convolution (the n-fold product per residue).
constexpr int kMaxInputs = 8;

// The twiddles of the stages live in one packed table per transform size:
// stage s, of radix R after Ns points have been combined (Ns > 1), reads the
// sub-table zeta_{Ns R}^e, e < Ns R, at toff[s]; its butterfly jm (< Ns)
// needs the entries r jm (r < R) and, in the twiddle-merged form, jm plus
// multiples of Ns R / 8.  A warp's butterflies so read neighbouring entries
// of a small table instead of entries r jm n / (Ns R) apart in the n-entry
// one.
struct FftPlan {
    int n;                          // transform size
    int nst;                        // number of stages
    int8_t rad[HDC_MAX_STAGES];     // radix per stage, product = n
    int32_t toff[HDC_MAX_STAGES];   // offset of the stage's twiddle sub-table
    int32_t tlen;                   // entries of the packed table (>= 1)
};

// ---------------------------------------------------------- one stage
// src -> dst (distinct shared buffers); one barrier at the end.
//
// With SWZ, logical element x lives at x ^ ((x / S) & (S - 1)), S = 128 /
// sizeof(V) elements per 128-byte bank row: the low bits are XORed with the
// row number, so the elements of one bank row stay in it but a run of
// elements with stride S (the first stage's outputs, R apart with R = 8)
// spreads over all banks.  Unlike a pad slot this keeps every buffer at its
// logical size.  The row buffers use it; the column tiles (ld = C, cs = 1)
// keep the plain layout, where neighbouring threads already take
// neighbouring columns and the index arithmetic measured slower.

// x / d for x >= 0, d > 0 without a runtime division where it can: a shift
// when d is a power of two, a 32-bit division when both fit in 31 bits (a
// 64-bit division costs several times the instructions of a 32-bit one,
// and both many times a shift).  The tests on d are the same for every
// thread of a launch.
__device__ __forceinline__ int div_idx(int x, int d)
{
    return (d & (d - 1)) == 0 ? (x >> (__ffs(d) - 1)) : x / d;
}
__device__ __forceinline__ int64_t div_idx(int64_t x, int64_t d)
{
    if ((d & (d - 1)) == 0) return x >> (__ffsll(d) - 1);
    if (((x | d) >> 31) == 0) return (int64_t)((unsigned)x / (unsigned)d);
    return x / d;
}

// (r t) mod q for the fold and unfold twiddles zeta_q^{r t}: the product in
// 64 bits, the remainder by a 32-bit division when the product fits
__device__ __forceinline__ int64_t rt_mod(int64_t r, int64_t t, int64_t q)
{
    const int64_t rt = r * t;
    if (((rt | q) >> 31) == 0) return (int64_t)((unsigned)rt % (unsigned)q);
    return rt % q;
}

template <class V, bool SWZ> __device__ __forceinline__ int sidx(int x)
{
    constexpr int S = 128 / (int)sizeof(V);
    return SWZ ? x ^ (int)(((unsigned)x / (unsigned)S) & (unsigned)(S - 1)) : x;
}

// shared-memory elements a buffer of n logical elements occupies (whole bank
// rows, so the swizzle stays inside it)
template <class V> __host__ __device__ constexpr int64_t smem_len(int64_t n)
{
    constexpr int64_t S = 128 / (int64_t)sizeof(V);
    return (n + S - 1) / S * S;
}

// tw / twl: the stage's sub-table zeta_{Ns R}^e (plain / twiddle-merged form).
// csh / nsh: log2 of ncol / Ns when it is a power of two, else -1 (the
// index arithmetic then takes shifts and masks instead of divisions, which
// cost about twenty integer instructions each per butterfly).
template <class V, int R, bool INV, bool SWZ, bool TS = false>
__device__ __forceinline__ void fft_stage(const V* src, V* dst, int n, int ncol, int ld, int cs, int Ns, int csh,
                                          int nsh, const V* __restrict__ tw, const V* __restrict__ twl, int tid,
                                          int nthr)
{
    constexpr bool kLF = (R == 2 || R == 4 || R == 8);
    const int nb = n / R;
    const int total = nb * ncol;
    for (int b = tid; b < total; b += nthr) {
        const int j = csh >= 0 ? (b >> csh) : b / ncol;
        const int c = b - j * ncol;
        const int base = c * cs;
        V v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[sidx<V, SWZ>(base + (j + r * nb) * ld)];
        const int jm = nsh >= 0 ? (j & (Ns - 1)) : j % Ns;
        if (kLF && Ns > 1) {
            // every butterfly of the stage carries its twiddles (W = 1 when jm = 0)
            DftLF<V, kLF ? R : 2, INV, TS>::run(v, twl, jm, Ns * R);
        } else if constexpr (R == 16) {
            if (jm != 0) {
                // four table entries w^1, w^2, w^4, w^8 (w = zeta_{Ns R}^jm)
                // and the other powers as their products: at most four
                // correctly rounded factors per twiddle, a quarter of the
                // table loads of one entry per input
                const V w1 = ld_tw<V, TS>(tw + jm), w2 = ld_tw<V, TS>(tw + 2 * jm);
                const V w4 = ld_tw<V, TS>(tw + 4 * jm), w8 = ld_tw<V, TS>(tw + 8 * jm);
                const V w3 = cmul(w1, w2), w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
                const V wp[8] = { czero<V>(), w1, w2, w3, w4, w5, w6, w7 };
#pragma unroll
                for (int r = 1; r < 8; ++r) v[r] = INV ? cmulc(v[r], wp[r]) : cmul(v[r], wp[r]);
                v[8] = INV ? cmulc(v[8], w8) : cmul(v[8], w8);
#pragma unroll
                for (int r = 9; r < 16; ++r) {
                    const V w = cmul(wp[r - 8], w8);
                    v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
                }
            }
            Dft<V, R, INV>::run(v);
        } else {
            if (jm != 0) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const V w = ld_tw<V, TS>(tw + r * jm);
                    v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
                }
            }
            Dft<V, R, INV>::run(v);
        }
        const int o = base + ((j - jm) * R + jm) * ld;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[sidx<V, SWZ>(o + r * Ns * ld)] = v[r];
    }
    __syncthreads();
}

// Whole transform of the ncol columns in buf, using tmp (same size and
// addressing) as the other half of the ping-pong.  tw / twl: the packed
// twiddle tables of fp (plain / twiddle-merged form, see FftPlan).  The
// caller must have synchronised after filling buf; the result is left where
// the last stage wrote it (buf after an even number of stages, tmp after an
// odd one), which is returned, and the block is synchronised.  R16: the
// kernel is built with the radix-16 stage (FP32 only); a plan that has one
// must be run with R16.  TS: tw and twl point to shared memory.
template <class V, bool INV, bool SWZ = false, bool R16 = false, bool TS = false>
__device__ __forceinline__ V* fft_smem_any(V* buf, V* tmp, const FftPlan& fp, int ncol, int ld, int cs,
                                           const V* __restrict__ tw, const V* __restrict__ twl, int tid, int nthr)
{
    int Ns = 1, nsh = 0;
    const int csh = (ncol & (ncol - 1)) == 0 ? __ffs(ncol) - 1 : -1;
    const int n = fp.n;
    V* a = buf;
    V* b = tmp;
    for (int s = 0; s < fp.nst; ++s) {
        const int R = fp.rad[s];
        const V* ts = tw + fp.toff[s];
        const V* tl = twl + fp.toff[s];
        switch (R) {
        case 16:  // FP32 plans only; compiled into the kernels that take them
            if constexpr (R16 && sizeof(V) == 8)
                fft_stage<V, 16, INV, SWZ, TS>(a, b, n, ncol, ld, cs, Ns, csh, nsh, ts, tl, tid, nthr);
            break;
        case 8: fft_stage<V, 8, INV, SWZ, TS>(a, b, n, ncol, ld, cs, Ns, csh, nsh, ts, tl, tid, nthr); break;
        case 4: fft_stage<V, 4, INV, SWZ, TS>(a, b, n, ncol, ld, cs, Ns, csh, nsh, ts, tl, tid, nthr); break;
        case 2: fft_stage<V, 2, INV, SWZ, TS>(a, b, n, ncol, ld, cs, Ns, csh, nsh, ts, tl, tid, nthr); break;
        case 3: fft_stage<V, 3, INV, SWZ, TS>(a, b, n, ncol, ld, cs, Ns, csh, nsh, ts, tl, tid, nthr); break;
        case 5: fft_stage<V, 5, INV, SWZ, TS>(a, b, n, ncol, ld, cs, Ns, csh, nsh, ts, tl, tid, nthr); break;
        case 7: fft_stage<V, 7, INV, SWZ, TS>(a, b, n, ncol, ld, cs, Ns, csh, nsh, ts, tl, tid, nthr); break;
        default: break;
        }
        Ns *= R;
        nsh = (nsh >= 0 && (R & (R - 1)) == 0) ? nsh + __ffs(R) - 1 : -1;
        V* t = a;
        a = b;
        b = t;
    }
    return a;
}

// The same with the result copied back into buf when it ended in tmp.
template <class V, bool INV, bool SWZ = false, bool R16 = false, bool TS = false>
__device__ __forceinline__ void fft_smem(V* buf, V* tmp, const FftPlan& fp, int ncol, int ld, int cs,
                                         const V* __restrict__ tw, const V* __restrict__ twl, int tid, int nthr)
{
    const V* a = fft_smem_any<V, INV, SWZ, R16, TS>(buf, tmp, fp, ncol, ld, cs, tw, twl, tid, nthr);
    if (a != buf) {
        const int tot = fp.n * ncol;
        for (int e = tid; e < tot; e += nthr) {
            const int i = div_idx(e, ncol), c = e - i * ncol;
            buf[sidx<V, SWZ>(c * cs + i * ld)] = a[sidx<V, SWZ>(c * cs + i * ld)];
        }
        __syncthreads();
    }
}

} // namespace hdc

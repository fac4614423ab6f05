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
// ever needed.  Twiddles come from a table tw[k] = zeta_n^k, k < n, made in
// FP64 from exact integer angles.
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
// a * w
template <class V> __device__ __forceinline__ V cmul(V a, V w)
{
    return mkc<V>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// a * conj(w)
template <class V> __device__ __forceinline__ V cmulc(V a, V w)
{
    return mkc<V>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y);
}
// acc + a * w
template <class V> __device__ __forceinline__ V cfma(V a, V w, V acc)
{
    return mkc<V>(acc.x + a.x * w.x - a.y * w.y, acc.y + a.x * w.y + a.y * w.x);
}
// acc + a * conj(w)
template <class V> __device__ __forceinline__ V cfmac(V a, V w, V acc)
{
    return mkc<V>(acc.x + a.x * w.x + a.y * w.y, acc.y + a.y * w.x - a.x * w.y);
}
// multiply by +i (forward) or -i (inverse)
template <class V, bool INV> __device__ __forceinline__ V rot90(V a)
{
    return INV ? mkc<V>(a.y, -a.x) : mkc<V>(-a.y, a.x);
}

template <class V> __device__ __forceinline__ V ldg_c(const V* p) { return __ldg(p); }

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
        // o_k *= zeta_8^{+-k}
        V w1, w3;
        if (!INV) {
            w1 = mkc<V>(h * (o1.x - o1.y), h * (o1.x + o1.y));
            w3 = mkc<V>(-h * (o3.x + o3.y), h * (o3.x - o3.y));
        } else {
            w1 = mkc<V>(h * (o1.x + o1.y), h * (o1.y - o1.x));
            w3 = mkc<V>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
        }
        V w2 = rot90<V, INV>(o2);
        v[0] = cadd(e0, o0);
        v[4] = csub(e0, o0);
        v[1] = cadd(e1, w1);
        v[5] = csub(e1, w1);
        v[2] = cadd(e2, w2);
        v[6] = csub(e2, w2);
        v[3] = cadd(e3, w3);
        v[7] = csub(e3, w3);
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

// ---------------------------------------------------------- FFT plan

#define HDC_MAX_STAGES 32

struct FftPlan {
    int n;                      // transform size
    int nst;                    // number of stages
    int8_t rad[HDC_MAX_STAGES]; // radix per stage, product = n
};

// ---------------------------------------------------------- one stage
// src -> dst (distinct shared buffers); one barrier at the end.

template <class V, int R, bool INV>
__device__ __forceinline__ void fft_stage(const V* src, V* dst, int n, int ncol, int ld, int cs, int Ns,
                                          const V* __restrict__ tw, int tid, int nthr)
{
    const int nb = n / R;
    const int total = nb * ncol;
    const int tstep = n / (Ns * R);
    for (int b = tid; b < total; b += nthr) {
        const int j = b / ncol;
        const int c = b - j * ncol;
        const int base = c * cs;
        V v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[base + (j + r * nb) * ld];
        const int jm = j % Ns;
        if (jm != 0) {
            const int k = jm * tstep;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const V w = ldg_c(tw + r * k);
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        Dft<V, R, INV>::run(v);
        const int o = base + ((j - jm) * R + jm) * ld;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[o + r * Ns * ld] = v[r];
    }
    __syncthreads();
}

// Whole transform of the ncol columns in buf, using tmp (same size and
// addressing) as the other half of the ping-pong.  The caller must have
// synchronised after filling buf; on return the result is in buf and the
// block is synchronised.
template <class V, bool INV>
__device__ __forceinline__ void fft_smem(V* buf, V* tmp, const FftPlan& fp, int ncol, int ld, int cs,
                                         const V* __restrict__ tw, int tid, int nthr)
{
    int Ns = 1;
    const int n = fp.n;
    V* a = buf;
    V* b = tmp;
    for (int s = 0; s < fp.nst; ++s) {
        const int R = fp.rad[s];
        switch (R) {
        case 8: fft_stage<V, 8, INV>(a, b, n, ncol, ld, cs, Ns, tw, tid, nthr); break;
        case 4: fft_stage<V, 4, INV>(a, b, n, ncol, ld, cs, Ns, tw, tid, nthr); break;
        case 2: fft_stage<V, 2, INV>(a, b, n, ncol, ld, cs, Ns, tw, tid, nthr); break;
        case 3: fft_stage<V, 3, INV>(a, b, n, ncol, ld, cs, Ns, tw, tid, nthr); break;
        case 5: fft_stage<V, 5, INV>(a, b, n, ncol, ld, cs, Ns, tw, tid, nthr); break;
        case 7: fft_stage<V, 7, INV>(a, b, n, ncol, ld, cs, Ns, tw, tid, nthr); break;
        default: break;
        }
        Ns *= R;
        V* t = a;
        a = b;
        b = t;
    }
    if (a != buf) {
        const int tot = n * ncol;
        for (int e = tid; e < tot; e += nthr) {
            const int i = e / ncol, c = e - i * ncol;
            buf[c * cs + i * ld] = a[c * cs + i * ld];
        }
        __syncthreads();
    }
}

} // namespace hdc

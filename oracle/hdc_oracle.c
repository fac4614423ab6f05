/*
 * hdc_oracle.c -- CPU oracle for hybrid dealiased convolution.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the bench may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Every routine is the plain, slow, obviously-correct form of what the paper
 * defines.  Complex arrays are interleaved (re, im) doubles, row-major with
 * the last axis fastest.
 *
 *   O1  direct linear convolution (Eq. 4), double-double accumulation
 *   O2  explicit zero-padded radix-2 FFT convolution (Section 2.4, the
 *       convolution theorem with explicit padding M >= 2L-1, Section 3.1)
 *   O3  exact integer convolution (int64 direct, or NTT mod 998244353)
 *   O4  closed forms of exponential and geometric sequences
 *   O5  residue forward/backward transforms written out as Eq. 1 and Eq. 2,
 *       and the hybrid convolution built from them (Section 2.2, 3.3, 3.5)
 *   O6  centered Hermitian (2-D) convolution by its definition
 *   O7  the parameter predictor's MLP: loss and gradients in FP64, Adam
 *   O8  unequal lengths with residue matching (Section 3.5, the final
 *       algorithm for one dimension), built from O5's Eq. 1 and Eq. 2
 *   O9  multi-convolution of n arrays: the n-fold convolution, or the sum
 *       of pairwise convolutions, by the same residue transforms
 *   O10 convolution of real inputs by the residue transforms of the packed
 *       sequence z = f + i g and the conjugate pairing of residues
 *
 * Sign convention (the paper's Eq. 1 and Eq. 2): zeta_n = exp(2 pi i / n),
 * forward transforms use zeta^{+kj} unscaled, backward use zeta^{-kj}/n.
 *
 * The convolution of length-L inputs keeps the first L outputs:
 *   h_k = sum_{j=0}^{k} f_j g_{k-j},  k = 0..L-1      (Eq. 4)
 * and per axis in N dimensions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HDCO_API __attribute__((visibility("default")))

/* ---------------------------------------------------------------- roots */

/* (cos, sin) of 2 pi k / n with k reduced in integers first and the angle
 * folded into [0, pi/4] so the libm argument is small and exact-ish. */
static void root_of_unity(int64_t k, int64_t n, double* c, double* s)
{
    k %= n;
    if (k < 0) k += n;
    /* use 8k against n to find the octant without rounding */
    int64_t k8 = 8 * k;
    double cc, ss;
    int neg_s = 0;
    /* map to upper half: angle in [0, pi] */
    if (2 * k > n) { k = n - k; neg_s = 1; k8 = 8 * k; }
    /* now angle = 2 pi k / n in [0, pi] */
    if (k8 <= n) {                       /* [0, pi/4] */
        double a = 2.0 * M_PI * ((double)k / (double)n);
        cc = cos(a); ss = sin(a);
    } else if (k8 <= 2 * n) {            /* (pi/4, pi/2]: use pi/2 - a */
        double a = 2.0 * M_PI * ((double)(n - 4 * k) / (4.0 * (double)n));
        cc = sin(a); ss = cos(a);
    } else if (k8 <= 3 * n) {            /* (pi/2, 3pi/4]: a - pi/2 */
        double a = 2.0 * M_PI * ((double)(4 * k - n) / (4.0 * (double)n));
        cc = -sin(a); ss = cos(a);
    } else {                             /* (3pi/4, pi]: pi - a */
        double a = 2.0 * M_PI * ((double)(n - 2 * k) / (2.0 * (double)n));
        cc = -cos(a); ss = sin(a);
    }
    *c = cc;
    *s = neg_s ? -ss : ss;
}

HDCO_API void hdco_root_of_unity(int64_t k, int64_t n, double* out2)
{
    root_of_unity(k, n, &out2[0], &out2[1]);
}

/* --------------------------------------------------------- double-double */

typedef struct { double hi, lo; } dd_t;

static inline dd_t two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    dd_t r = { s, e };
    return r;
}

static inline dd_t dd_add_d(dd_t x, double y)
{
    dd_t s = two_sum(x.hi, y);
    double lo = s.lo + x.lo;
    dd_t r = two_sum(s.hi, lo);
    return r;
}

/* x += a*b exactly-rounded into the double-double accumulator */
static inline dd_t dd_fma_acc(dd_t x, double a, double b)
{
    double p = a * b;
    double e = fma(a, b, -p);
    x = dd_add_d(x, p);
    return dd_add_d(x, e);
}

/* ------------------------------------------------------------ O1 direct */

/* One output of the N-D direct convolution, dims padded to 3 with 1s.
 * h[k0,k1,k2] = sum_{j0<=k0, j1<=k1, j2<=k2} f[j] g[k-j]. */
static void direct_point(const double* f, const double* g, const int64_t L[3],
                         int64_t k0, int64_t k1, int64_t k2, double* out2)
{
    dd_t re = { 0.0, 0.0 }, im = { 0.0, 0.0 };
    for (int64_t j0 = 0; j0 <= k0; ++j0)
        for (int64_t j1 = 0; j1 <= k1; ++j1) {
            const double* fr = f + 2 * ((j0 * L[1] + j1) * L[2]);
            const double* gr = g + 2 * (((k0 - j0) * L[1] + (k1 - j1)) * L[2]);
            for (int64_t j2 = 0; j2 <= k2; ++j2) {
                double a = fr[2 * j2], b = fr[2 * j2 + 1];
                double c = gr[2 * (k2 - j2)], d = gr[2 * (k2 - j2) + 1];
                re = dd_fma_acc(re, a, c);
                re = dd_fma_acc(re, -b, d);
                im = dd_fma_acc(im, a, d);
                im = dd_fma_acc(im, b, c);
            }
        }
    out2[0] = re.hi + re.lo;
    out2[1] = im.hi + im.lo;
}

static void dims3(int dims, const int64_t* L, int64_t out[3])
{
    out[0] = out[1] = out[2] = 1;
    for (int i = 0; i < dims; ++i) out[3 - dims + i] = L[i];
}

/* Direct convolution, first L outputs per axis, dims in {1,2,3}. */
HDCO_API int hdco_conv_direct(int dims, const int64_t* Ld, const double* f,
                              const double* g, double* h)
{
    if (dims < 1 || dims > 3) return -1;
    int64_t L[3];
    dims3(dims, Ld, L);
    int64_t total = L[0] * L[1] * L[2];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t idx = total - 1; idx >= 0; --idx) {
        int64_t k2 = idx % L[2];
        int64_t k1 = (idx / L[2]) % L[1];
        int64_t k0 = idx / (L[1] * L[2]);
        direct_point(f, g, L, k0, k1, k2, h + 2 * idx);
    }
    return 0;
}

/* Direct convolution at selected flat output indices only (sampled check of
 * full-size outputs). */
HDCO_API int hdco_conv_direct_at(int dims, const int64_t* Ld, const double* f,
                                 const double* g, const int64_t* idx,
                                 int64_t nidx, double* out)
{
    if (dims < 1 || dims > 3) return -1;
    int64_t L[3];
    dims3(dims, Ld, L);
    int64_t total = L[0] * L[1] * L[2];
    for (int64_t i = 0; i < nidx; ++i)
        if (idx[i] < 0 || idx[i] >= total) return -2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < nidx; ++i) {
        int64_t id = idx[i];
        int64_t k2 = id % L[2];
        int64_t k1 = (id / L[2]) % L[1];
        int64_t k0 = id / (L[1] * L[2]);
        direct_point(f, g, L, k0, k1, k2, out + 2 * i);
    }
    return 0;
}

/* ---------------------------------------------------- O2 explicit FFT */

/* In-place iterative radix-2 FFT of n = 2^k points with stride between
 * points (in complex elements).  sign=+1: sum zeta^{+kj}; -1: zeta^{-kj}.
 * No scaling. */
static void fft_radix2(double* a, int64_t n, int64_t stride, int sign,
                       const double* roots /* roots[2k] = zeta_n^k, k<n/2 */)
{
    /* bit reversal */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double* x = a + 2 * i * stride;
            double* y = a + 2 * j * stride;
            double t0 = x[0], t1 = x[1];
            x[0] = y[0]; x[1] = y[1];
            y[0] = t0; y[1] = t1;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1;
        int64_t step = n / len;
        for (int64_t i = 0; i < n; i += len)
            for (int64_t k = 0; k < half; ++k) {
                double wr = roots[2 * k * step];
                double wi = sign * roots[2 * k * step + 1];
                double* u = a + 2 * (i + k) * stride;
                double* v = a + 2 * (i + k + half) * stride;
                double vr = v[0] * wr - v[1] * wi;
                double vi = v[0] * wi + v[1] * wr;
                v[0] = u[0] - vr; v[1] = u[1] - vi;
                u[0] += vr; u[1] += vi;
            }
    }
}

static int64_t pow2_at_least(int64_t n)
{
    int64_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

/* N-D transform of a padded array P[0..N0)[0..N1)[0..N2) along every axis
 * with extent > 1. */
static void fft_nd(double* P, const int64_t N[3], int sign)
{
    for (int ax = 0; ax < 3; ++ax) {
        int64_t n = N[ax];
        if (n == 1) continue;
        double* roots = (double*)malloc(sizeof(double) * (size_t)n);
        for (int64_t k = 0; k < n / 2; ++k) root_of_unity(k, n, &roots[2 * k], &roots[2 * k + 1]);
        int64_t stride = (ax == 0) ? N[1] * N[2] : (ax == 1 ? N[2] : 1);
        int64_t nlines = (N[0] * N[1] * N[2]) / n;
#pragma omp parallel for schedule(static)
        for (int64_t line = 0; line < nlines; ++line) {
            int64_t base;
            if (ax == 0) base = line;                       /* (i1, i2) */
            else if (ax == 1) base = (line / N[2]) * N[1] * N[2] + (line % N[2]);
            else base = line * N[2];
            fft_radix2(P + 2 * base, n, stride, sign, roots);
        }
        free(roots);
    }
}

/* Explicitly padded FFT convolution: pad each axis to 2^ceil(log2(2L-1)),
 * transform, multiply, inverse transform, scale, keep the first L per axis. */
HDCO_API int hdco_conv_fft(int dims, const int64_t* Ld, const double* f,
                           const double* g, double* h)
{
    if (dims < 1 || dims > 3) return -1;
    int64_t L[3], N[3];
    dims3(dims, Ld, L);
    for (int i = 0; i < 3; ++i) N[i] = (L[i] == 1) ? 1 : pow2_at_least(2 * L[i] - 1);
    int64_t tot = N[0] * N[1] * N[2];
    double* A = (double*)calloc((size_t)(2 * tot), sizeof(double));
    double* B = (double*)calloc((size_t)(2 * tot), sizeof(double));
    if (!A || !B) { free(A); free(B); return -3; }
    for (int64_t i0 = 0; i0 < L[0]; ++i0)
        for (int64_t i1 = 0; i1 < L[1]; ++i1) {
            int64_t src = (i0 * L[1] + i1) * L[2];
            int64_t dst = (i0 * N[1] + i1) * N[2];
            memcpy(A + 2 * dst, f + 2 * src, sizeof(double) * 2 * (size_t)L[2]);
            memcpy(B + 2 * dst, g + 2 * src, sizeof(double) * 2 * (size_t)L[2]);
        }
    fft_nd(A, N, +1);
    fft_nd(B, N, +1);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < tot; ++i) {
        double a = A[2 * i], b = A[2 * i + 1], c = B[2 * i], d = B[2 * i + 1];
        A[2 * i] = a * c - b * d;
        A[2 * i + 1] = a * d + b * c;
    }
    fft_nd(A, N, -1);
    double scale = 1.0 / (double)tot;
    for (int64_t i0 = 0; i0 < L[0]; ++i0)
        for (int64_t i1 = 0; i1 < L[1]; ++i1)
            for (int64_t i2 = 0; i2 < L[2]; ++i2) {
                int64_t src = (i0 * N[1] + i1) * N[2] + i2;
                int64_t dst = (i0 * L[1] + i1) * L[2] + i2;
                h[2 * dst] = A[2 * src] * scale;
                h[2 * dst + 1] = A[2 * src + 1] * scale;
            }
    free(A);
    free(B);
    return 0;
}

/* Plain DFT by definition, X_k = sum_j zeta_n^{sign k j} x_j (test helper for
 * pinning the FFT on non-power-of-two lengths is not needed; this one pins
 * the residue transforms on tiny sizes). */
HDCO_API void hdco_dft(const double* x, int64_t n, int sign, double* X)
{
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double c, s;
            root_of_unity((k * j) % n, n, &c, &s);
            s *= sign;
            sr += x[2 * j] * c - x[2 * j + 1] * s;
            si += x[2 * j] * s + x[2 * j + 1] * c;
        }
        X[2 * k] = sr;
        X[2 * k + 1] = si;
    }
}

/* ------------------------------------------------------ O3 exact integer */

#define NTT_P 998244353ULL
#define NTT_G 3ULL

static uint64_t pow_mod(uint64_t b, uint64_t e)
{
    uint64_t r = 1;
    b %= NTT_P;
    while (e) {
        if (e & 1) r = r * b % NTT_P;
        b = b * b % NTT_P;
        e >>= 1;
    }
    return r;
}

static void ntt(uint64_t* a, int64_t n, int invert)
{
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        uint64_t w = pow_mod(NTT_G, (NTT_P - 1) / (uint64_t)len);
        if (invert) w = pow_mod(w, NTT_P - 2);
        int64_t half = len >> 1;
        /* powers of w for this stage */
        uint64_t* wp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)half);
        wp[0] = 1;
        for (int64_t k = 1; k < half; ++k) wp[k] = wp[k - 1] * w % NTT_P;
#pragma omp parallel for schedule(static) if (n >= 65536)
        for (int64_t i = 0; i < n; i += len)
            for (int64_t k = 0; k < half; ++k) {
                uint64_t u = a[i + k];
                uint64_t v = a[i + k + half] * wp[k] % NTT_P;
                a[i + k] = (u + v) % NTT_P;
                a[i + k + half] = (u + NTT_P - v) % NTT_P;
            }
        free(wp);
    }
    if (invert) {
        uint64_t ninv = pow_mod((uint64_t)n, NTT_P - 2);
        for (int64_t i = 0; i < n; ++i) a[i] = a[i] * ninv % NTT_P;
    }
}

static int64_t lift(uint64_t v)
{
    return (v > NTT_P / 2) ? (int64_t)v - (int64_t)NTT_P : (int64_t)v;
}

/* First L outputs of the real linear convolution of integer a, c.  Each
 * |output| must stay below P/2 (true for |a|,|c| <= 8 and L <= 2^22). */
static int int_conv_real(const int64_t* a, const int64_t* c, int64_t L, int64_t* out, int use_ntt)
{
    if (!use_ntt) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t k = 0; k < L; ++k) {
            int64_t s = 0;
            for (int64_t j = 0; j <= k; ++j) s += a[j] * c[k - j];
            out[k] = s;
        }
        return 0;
    }
    int64_t n = pow2_at_least(2 * L - 1);
    if (n > (1LL << 23)) return -4;
    uint64_t* A = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    uint64_t* C = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    if (!A || !C) { free(A); free(C); return -3; }
    for (int64_t i = 0; i < L; ++i) {
        A[i] = (uint64_t)((a[i] % (int64_t)NTT_P + (int64_t)NTT_P) % (int64_t)NTT_P);
        C[i] = (uint64_t)((c[i] % (int64_t)NTT_P + (int64_t)NTT_P) % (int64_t)NTT_P);
    }
    ntt(A, n, 0);
    ntt(C, n, 0);
    for (int64_t i = 0; i < n; ++i) A[i] = A[i] * C[i] % NTT_P;
    ntt(A, n, 1);
    for (int64_t k = 0; k < L; ++k) out[k] = lift(A[k]);
    free(A);
    free(C);
    return 0;
}

/* Complex integer convolution (a+ib)*(c+id): four real convolutions.
 * method: 0 = int64 direct, 1 = NTT. */
HDCO_API int hdco_conv_int_exact_1d(const int64_t* fre, const int64_t* fim,
                                    const int64_t* gre, const int64_t* gim,
                                    int64_t L, int method, int64_t* hre,
                                    int64_t* him)
{
    int64_t* t1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
    int64_t* t2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
    if (!t1 || !t2) { free(t1); free(t2); return -3; }
    int rc = 0;
    rc |= int_conv_real(fre, gre, L, t1, method);   /* ac */
    rc |= int_conv_real(fim, gim, L, t2, method);   /* bd */
    for (int64_t k = 0; k < L; ++k) hre[k] = t1[k] - t2[k];
    rc |= int_conv_real(fre, gim, L, t1, method);   /* ad */
    rc |= int_conv_real(fim, gre, L, t2, method);   /* bc */
    for (int64_t k = 0; k < L; ++k) him[k] = t1[k] + t2[k];
    free(t1);
    free(t2);
    return rc;
}

/* ---------------------------------------------------------- O4 closed forms */

static void cmul(double a, double b, double c, double d, double* re, double* im)
{
    *re = a * c - b * d;
    *im = a * d + b * c;
}

/* f_j = zeta_P^{A j}, g_j = zeta_P^{B j}.  Then
 *   h_k = zeta_P^{B k} sum_{j=0}^{k} zeta_P^{(A-B) j}
 *       = (k+1) zeta_P^{B k}                                  if A = B mod P
 *       = zeta_P^{B k} (1 - zeta_P^{(A-B)(k+1)}) / (1 - zeta_P^{A-B}) otherwise
 * (geometric series).  Exponents are reduced mod P in integers. */
HDCO_API void hdco_closed_form_exp_1d(int64_t A, int64_t B, int64_t P, int64_t L, double* h)
{
    int64_t D = ((A - B) % P + P) % P;
    double dc, ds;
    root_of_unity(D, P, &dc, &ds);
    double den_r = 1.0 - dc, den_i = -ds;
    double den2 = den_r * den_r + den_i * den_i;
    for (int64_t k = 0; k < L; ++k) {
        double bc, bs;
        root_of_unity(((B % P) * (k % P)) % P, P, &bc, &bs);
        if (D == 0) {
            h[2 * k] = (double)(k + 1) * bc;
            h[2 * k + 1] = (double)(k + 1) * bs;
            continue;
        }
        double nc, ns;
        root_of_unity((D * ((k + 1) % P)) % P, P, &nc, &ns);
        double num_r = 1.0 - nc, num_i = -ns;
        /* num / den */
        double qr = (num_r * den_r + num_i * den_i) / den2;
        double qi = (num_i * den_r - num_r * den_i) / den2;
        cmul(bc, bs, qr, qi, &h[2 * k], &h[2 * k + 1]);
    }
}

/* f_j = alpha^j, g_j = beta^j with alpha = ra zeta_P^{A}, beta = rb zeta_P^{B}
 * and alpha != beta:  h_k = (alpha^{k+1} - beta^{k+1}) / (alpha - beta). */
HDCO_API void hdco_closed_form_geom_1d(double ra, int64_t A, double rb, int64_t B,
                                       int64_t P, int64_t L, double* h)
{
    double ac, as, bc, bs;
    root_of_unity(A, P, &ac, &as);
    root_of_unity(B, P, &bc, &bs);
    double dr = ra * ac - rb * bc, di = ra * as - rb * bs;
    double d2 = dr * dr + di * di;
    for (int64_t k = 0; k < L; ++k) {
        double c1, s1, c2, s2;
        root_of_unity((A % P) * ((k + 1) % P) % P, P, &c1, &s1);
        root_of_unity((B % P) * ((k + 1) % P) % P, P, &c2, &s2);
        double m1 = pow(ra, (double)(k + 1)), m2 = pow(rb, (double)(k + 1));
        double nr = m1 * c1 - m2 * c2, ni = m1 * s1 - m2 * s2;
        h[2 * k] = (nr * dr + ni * di) / d2;
        h[2 * k + 1] = (ni * dr - nr * di) / d2;
    }
}

/* ------------------------------------------------ O5 residue transforms */

/* Eq. 1: for r < q, l < m,
 *   F_{q l + r} = sum_{s<m} zeta_m^{l s} zeta_{qm}^{r s} sum_{t<p} zeta_q^{r t} x_{t m + s}
 * with x_j = 0 for j >= L.  Output in natural order, N = q m entries. */
HDCO_API int hdco_residue_forward_1d(const double* x, int64_t L, int64_t m,
                                     int64_t p, int64_t q, double* F)
{
    if (m < 1 || p < 1 || q < 1 || p * m < L) return -1;
    int64_t N = q * m;
    double* w = (double*)malloc(sizeof(double) * 2 * (size_t)m);
    if (!w) return -3;
    for (int64_t r = 0; r < q; ++r) {
        /* inner sum over t, then the twiddle zeta_{qm}^{r s} */
        for (int64_t s = 0; s < m; ++s) {
            double ar = 0.0, ai = 0.0;
            for (int64_t t = 0; t < p; ++t) {
                int64_t j = t * m + s;
                if (j >= L) continue;
                double c, sn;
                root_of_unity((r * t) % q, q, &c, &sn);
                ar += x[2 * j] * c - x[2 * j + 1] * sn;
                ai += x[2 * j] * sn + x[2 * j + 1] * c;
            }
            double c, sn;
            root_of_unity((r * s) % N, N, &c, &sn);
            w[2 * s] = ar * c - ai * sn;
            w[2 * s + 1] = ar * sn + ai * c;
        }
        /* outer sum over s with zeta_m^{l s} */
        for (int64_t l = 0; l < m; ++l) {
            double sr = 0.0, si = 0.0;
            for (int64_t s = 0; s < m; ++s) {
                double c, sn;
                root_of_unity((l * s) % m, m, &c, &sn);
                sr += w[2 * s] * c - w[2 * s + 1] * sn;
                si += w[2 * s] * sn + w[2 * s + 1] * c;
            }
            F[2 * (q * l + r)] = sr;
            F[2 * (q * l + r) + 1] = si;
        }
    }
    free(w);
    return 0;
}

/* Eq. 2: for t < p, s < m with t m + s < L,
 *   x_{t m + s} = (1/(q m)) sum_{r<q} zeta_q^{-t r} zeta_{qm}^{-s r} sum_{l<m} zeta_m^{-s l} F_{q l + r}. */
HDCO_API int hdco_residue_backward_1d(const double* F, int64_t L, int64_t m,
                                      int64_t p, int64_t q, double* x)
{
    if (m < 1 || p < 1 || q < 1 || p * m < L) return -1;
    int64_t N = q * m;
    double* u = (double*)malloc(sizeof(double) * 2 * (size_t)(q * m));
    if (!u) return -3;
    /* u[r][s] = sum_l zeta_m^{-s l} F_{q l + r} */
    for (int64_t r = 0; r < q; ++r)
        for (int64_t s = 0; s < m; ++s) {
            double sr = 0.0, si = 0.0;
            for (int64_t l = 0; l < m; ++l) {
                double c, sn;
                root_of_unity((l * s) % m, m, &c, &sn);
                sn = -sn;
                const double* Fk = F + 2 * (q * l + r);
                sr += Fk[0] * c - Fk[1] * sn;
                si += Fk[0] * sn + Fk[1] * c;
            }
            u[2 * (r * m + s)] = sr;
            u[2 * (r * m + s) + 1] = si;
        }
    for (int64_t t = 0; t < p; ++t)
        for (int64_t s = 0; s < m; ++s) {
            int64_t j = t * m + s;
            if (j >= L) continue;
            double sr = 0.0, si = 0.0;
            for (int64_t r = 0; r < q; ++r) {
                double c1, s1, c2, s2;
                root_of_unity((t * r) % q, q, &c1, &s1);
                root_of_unity((s * r) % N, N, &c2, &s2);
                /* zeta_q^{-tr} zeta_{qm}^{-sr} */
                double wr = c1 * c2 - s1 * s2, wi = -(c1 * s2 + s1 * c2);
                const double* ur = u + 2 * (r * m + s);
                sr += ur[0] * wr - ur[1] * wi;
                si += ur[0] * wi + ur[1] * wr;
            }
            x[2 * j] = sr / (double)N;
            x[2 * j + 1] = si / (double)N;
        }
    free(u);
    return 0;
}

/* The hybrid convolution in the paper's order: Eq. 1 on f and g, pointwise
 * product of the q m transformed values, Eq. 2, first L outputs.  Requires
 * q m >= 2L - 1 (Section 3.1) for the result to be alias-free. */
HDCO_API int hdco_conv_hybrid_1d(const double* f, const double* g, int64_t L,
                                 int64_t m, int64_t p, int64_t q, double* h)
{
    int64_t N = q * m;
    double* F = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double* G = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!F || !G) { free(F); free(G); return -3; }
    int rc = hdco_residue_forward_1d(f, L, m, p, q, F);
    rc |= hdco_residue_forward_1d(g, L, m, p, q, G);
    if (rc) { free(F); free(G); return rc; }
    for (int64_t k = 0; k < N; ++k) {
        double a = F[2 * k], b = F[2 * k + 1], c = G[2 * k], d = G[2 * k + 1];
        F[2 * k] = a * c - b * d;
        F[2 * k + 1] = a * d + b * c;
    }
    rc = hdco_residue_backward_1d(F, L, m, p, q, h);
    free(F);
    free(G);
    return rc;
}

/* ------------------------------------------ O8 unequal lengths, 1-D */

/* Convolution of f (length Lf) and g (length Lg) by the final algorithm of
 * Section 3.5: f is transformed at m points, g at Lam m points,
 *   pf = ceil(Lf / m), pg = ceil(Lg / (Lam m)), qg = ceil(M / (Lam m)),
 *   qf = Lam qg,  N = qg Lam m = qf m.
 * The forward transforms are Eq. 1 for each input with its own (m, p, q)
 * (O5; entry q l + r holds residue r at bin l).  For each residue rg of g
 * and each Lam index l in [0, Lam), the matching residue of f is
 * rf = qg l + rg, and bin lg = Lam lf + l of residue rg of g multiplies bin
 * lf of residue rf of f (qg lg + rg = qf lf + rf).  The backward transform
 * is Eq. 2 with g's parameters, kept for outputs [o, o + Lw) of the linear
 * convolution.  Needs M >= Lf + Lg - 1 - o and o + Lw <= N (no aliasing).
 * Returns 0, or -1 on invalid parameters, -3 on allocation failure. */
HDCO_API int hdco_conv_unequal_1d(const double* f, int64_t Lf, const double* g, int64_t Lg,
                                  int64_t m, int64_t Lam, int64_t M, int64_t o, int64_t Lw,
                                  double* h)
{
    if (Lf < 1 || Lg < 1 || m < 1 || Lam < 1 || o < 0 || Lw < 1) return -1;
    if (M < Lf + Lg - 1 - o || o + Lw > Lf + Lg - 1) return -1;
    const int64_t mg = Lam * m;
    const int64_t pf = (Lf + m - 1) / m, pg = (Lg + mg - 1) / mg;
    const int64_t qg = (M + mg - 1) / mg, qf = Lam * qg;
    const int64_t N = qg * mg;
    if (o + Lw > N) return -1;
    const int64_t Lout = o + Lw, pout = (Lout + mg - 1) / mg;
    double* F = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double* G = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double* H = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double* x = (double*)malloc(sizeof(double) * 2 * (size_t)Lout);
    if (!F || !G || !H || !x) { free(F); free(G); free(H); free(x); return -3; }
    int rc = hdco_residue_forward_1d(f, Lf, m, pf, qf, F);
    rc |= hdco_residue_forward_1d(g, Lg, mg, pg, qg, G);
    if (rc) { free(F); free(G); free(H); free(x); return -1; }
    for (int64_t rg = 0; rg < qg; ++rg)
        for (int64_t l = 0; l < Lam; ++l) {
            const int64_t rf = qg * l + rg;
            for (int64_t lf = 0; lf < m; ++lf) {
                const int64_t lg = Lam * lf + l;
                const double* a = G + 2 * (qg * lg + rg);
                const double* b = F + 2 * (qf * lf + rf);
                double* c = H + 2 * (qg * lg + rg);
                c[0] = a[0] * b[0] - a[1] * b[1];
                c[1] = a[0] * b[1] + a[1] * b[0];
            }
        }
    rc = hdco_residue_backward_1d(H, Lout, mg, pout, qg, x);
    if (rc == 0) memcpy(h, x + 2 * o, sizeof(double) * 2 * (size_t)Lw);
    free(F); free(G); free(H); free(x);
    return rc ? -1 : 0;
}

/* ------------------------------------------- O9 multi-convolution, 1-D */

/* First L outputs of a multi-convolution of n length-L inputs
 * (concatenated in xs, input i at xs + 2 i L) by the residue transforms:
 * Eq. 1 for every input with the same (m, p, q); at every DFT index either
 * the product of all n transforms (op 0: the n-fold convolution
 * x_0 * x_1 * ... * x_{n-1}, full length n (L - 1) + 1, alias-free when
 * q m >= n (L - 1) + 1) or the sum of the pairwise products
 * F_0 F_1 + F_2 F_3 + ... (op 1, n even: x_0 * x_1 + x_2 * x_3 + ...,
 * alias-free when q m >= 2 L - 1); then Eq. 2.  Returns 0, -1 on invalid
 * parameters, -3 on allocation failure. */
HDCO_API int hdco_conv_multi_1d(const double* xs, int n, int op, int64_t L, int64_t m, int64_t p, int64_t q,
                                double* h)
{
    if (n < 1 || L < 1 || m < 1 || p * m < L || q < 1 || (op != 0 && op != 1)) return -1;
    if (op == 1 && (n % 2)) return -1;
    const int64_t N = q * m;
    const int64_t span = op == 0 ? (int64_t)n * (L - 1) + 1 : 2 * L - 1;
    if (N < span) return -1;
    double* H = (double*)calloc(2 * (size_t)N, sizeof(double));
    double* A = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double* F = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    if (!H || !A || !F) { free(H); free(A); free(F); return -3; }
    int rc = 0;
    if (op == 0) {
        rc = hdco_residue_forward_1d(xs, L, m, p, q, H);
        for (int i = 1; i < n && rc == 0; ++i) {
            rc = hdco_residue_forward_1d(xs + 2 * (size_t)i * (size_t)L, L, m, p, q, F);
            for (int64_t k = 0; k < N && rc == 0; ++k) {
                const double a = H[2 * k], b = H[2 * k + 1], c = F[2 * k], d = F[2 * k + 1];
                H[2 * k] = a * c - b * d;
                H[2 * k + 1] = a * d + b * c;
            }
        }
    } else {
        for (int i = 0; i + 1 < n && rc == 0; i += 2) {
            rc = hdco_residue_forward_1d(xs + 2 * (size_t)i * (size_t)L, L, m, p, q, A);
            rc |= hdco_residue_forward_1d(xs + 2 * (size_t)(i + 1) * (size_t)L, L, m, p, q, F);
            for (int64_t k = 0; k < N && rc == 0; ++k) {
                const double a = A[2 * k], b = A[2 * k + 1], c = F[2 * k], d = F[2 * k + 1];
                H[2 * k] += a * c - b * d;
                H[2 * k + 1] += a * d + b * c;
            }
        }
    }
    if (rc == 0) rc = hdco_residue_backward_1d(H, L, m, p, q, h);
    free(H);
    free(A);
    free(F);
    return rc ? -1 : 0;
}

/* ------------------------------------------ O10 real inputs, 1-D */

/* First L outputs of the convolution of real f and g (length L) through the
 * residue transforms of the complex sequence z = f + i g (Eq. 1 with
 * (m, p, q)).  Since f and g are real, F and G at DFT index K follow from Z
 * at K and N - K:  F_K = (Z_K + conj Z_{N-K}) / 2,  G_K = (Z_K - conj Z_{N-K})
 * / (2 i).  With K = q l + r, the index N - K lies in residue r' = (q - r)
 * mod q at bin (m - l) mod m when r = 0 and m - 1 - l otherwise.  Only the
 * residues r <= q / 2 are formed; the backward transform (Eq. 2) of residue
 * r' is the complex conjugate of that of r, so each output is the real part
 * of the residue-r contributions, doubled when r' != r.  Returns 0, or -1 on
 * invalid parameters (q m < 2 L - 1 included), -3 on allocation failure. */
HDCO_API int hdco_conv_real_1d(const double* f, const double* g, int64_t L, int64_t m, int64_t p, int64_t q,
                               double* h)
{
    if (L < 1 || m < 1 || p * m < L || q < 1 || q * m < 2 * L - 1) return -1;
    const int64_t N = q * m;
    double* z = (double*)malloc(sizeof(double) * 2 * (size_t)L);
    double* Z = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double* H = (double*)malloc(sizeof(double) * 2 * (size_t)N);
    double* x = (double*)malloc(sizeof(double) * 2 * (size_t)L);
    if (!z || !Z || !H || !x) { free(z); free(Z); free(H); free(x); return -3; }
    for (int64_t j = 0; j < L; ++j) { z[2 * j] = f[j]; z[2 * j + 1] = g[j]; }
    int rc = hdco_residue_forward_1d(z, L, m, p, q, Z);
    memset(H, 0, sizeof(double) * 2 * (size_t)N);
    for (int64_t r = 0; 2 * r <= q && rc == 0; ++r) {
        const int64_t rp = (q - r) % q;
        for (int64_t l = 0; l < m; ++l) {
            const int64_t lp = r == 0 ? (m - l) % m : m - 1 - l;
            const double* a = Z + 2 * (q * l + r);
            const double* b = Z + 2 * (q * lp + rp);
            /* F = (a + conj b) / 2, G = (a - conj b) / (2 i) */
            const double Fr = 0.5 * (a[0] + b[0]), Fi = 0.5 * (a[1] - b[1]);
            const double Dr = 0.5 * (a[0] - b[0]), Di = 0.5 * (a[1] + b[1]);
            const double Gr = Di, Gi = -Dr;
            double* c = H + 2 * (q * l + r);
            c[0] = Fr * Gr - Fi * Gi;
            c[1] = Fr * Gi + Fi * Gr;
        }
    }
    /* Eq. 2 over the kept residues only, weighted: residue r stands for
     * itself and, when r' != r, for its conjugate partner */
    for (int64_t j = 0; j < L && rc == 0; ++j) {
        const int64_t t = j / m, s = j % m;
        double acc = 0.0;
        for (int64_t r = 0; 2 * r <= q; ++r) {
            const int64_t rp = (q - r) % q;
            const double w = rp == r ? 1.0 : 2.0;
            /* u = sum_l zeta_m^{-s l} H_{q l + r}; term = zeta_q^{-t r} zeta_N^{-s r} u */
            double ur = 0.0, ui = 0.0;
            for (int64_t l = 0; l < m; ++l) {
                double cc, sn;
                root_of_unity((l * s) % m, m, &cc, &sn);
                sn = -sn;
                const double* Hk = H + 2 * (q * l + r);
                ur += Hk[0] * cc - Hk[1] * sn;
                ui += Hk[0] * sn + Hk[1] * cc;
            }
            double c1, s1, c2, s2;
            root_of_unity((t * r) % q, q, &c1, &s1);
            root_of_unity((s * r) % N, N, &c2, &s2);
            const double wr = c1 * c2 - s1 * s2, wi = -(c1 * s2 + s1 * c2);
            acc += w * (ur * wr - ui * wi);
        }
        x[2 * j] = acc / (double)N;
    }
    if (rc == 0)
        for (int64_t j = 0; j < L; ++j) h[j] = x[2 * j];
    free(z); free(Z); free(H); free(x);
    return rc ? -1 : 0;
}

/* ------------------------------------------- O6 centered Hermitian 2-D */

/* Centered 2-D convolution on the box |kx|, |ky| <= K-1 of two spectra given
 * by their non-redundant halves (rows kx = -(K-1)..K-1, columns ky = 0..K-1;
 * the other half is the complex conjugate, f(-k) = conj(f(k))):
 *   h_k = sum_{p, k-p in box} f_p g_{k-p},  k in the box, ky >= 0.
 * Output in the same (2K-1) x K layout. Direct O(K^4): tiny K only. */
static void herm_get(const double* a, int64_t K, int64_t kx, int64_t ky, double* re, double* im)
{
    int64_t c = K - 1;
    if (ky >= 0) {
        const double* v = a + 2 * ((kx + c) * K + ky);
        *re = v[0]; *im = v[1];
    } else {
        const double* v = a + 2 * ((-kx + c) * K + (-ky));
        *re = v[0]; *im = -v[1];
    }
}

HDCO_API int hdco_conv_hermitian_2d_direct(const double* f, const double* g,
                                           int64_t K, double* h)
{
    int64_t c = K - 1;
    int64_t nx = 2 * K - 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ix = 0; ix < nx; ++ix) {
        int64_t kx = ix - c;
        for (int64_t ky = 0; ky < K; ++ky) {
            dd_t re = { 0.0, 0.0 }, im = { 0.0, 0.0 };
            for (int64_t px = -c; px <= c; ++px) {
                int64_t qx = kx - px;
                if (qx < -c || qx > c) continue;
                for (int64_t py = -c; py <= c; ++py) {
                    int64_t qy = ky - py;
                    if (qy < -c || qy > c) continue;
                    double a, b, cc, d;
                    herm_get(f, K, px, py, &a, &b);
                    herm_get(g, K, qx, qy, &cc, &d);
                    re = dd_fma_acc(re, a, cc);
                    re = dd_fma_acc(re, -b, d);
                    im = dd_fma_acc(im, a, d);
                    im = dd_fma_acc(im, b, cc);
                }
            }
            h[2 * (ix * K + ky)] = re.hi + re.lo;
            h[2 * (ix * K + ky) + 1] = im.hi + im.lo;
        }
    }
    return 0;
}

/* The same centered Hermitian convolution by explicit zero padding: build the
 * full (2K-1)^2 centered spectra, place them in an n x n periodic grid with
 * n = 2^ceil(log2(4K-3)) (alias-free for the centered sum), transform back
 * to physical space, multiply, transform forward, read the box. */
HDCO_API int hdco_conv_hermitian_2d_fft(const double* f, const double* g,
                                        int64_t K, double* h)
{
    int64_t c = K - 1;
    int64_t n = pow2_at_least(4 * K - 3);
    int64_t N[3] = { 1, n, n };
    double* A = (double*)calloc((size_t)(2 * n * n), sizeof(double));
    double* B = (double*)calloc((size_t)(2 * n * n), sizeof(double));
    if (!A || !B) { free(A); free(B); return -3; }
    for (int64_t kx = -c; kx <= c; ++kx)
        for (int64_t ky = -c; ky <= c; ++ky) {
            int64_t ix = (kx + n) % n, iy = (ky + n) % n;
            herm_get(f, K, kx, ky, &A[2 * (ix * n + iy)], &A[2 * (ix * n + iy) + 1]);
            herm_get(g, K, kx, ky, &B[2 * (ix * n + iy)], &B[2 * (ix * n + iy) + 1]);
        }
    /* to physical space: u(x) = sum_k f_k zeta^{k x} */
    fft_nd(A, N, +1);
    fft_nd(B, N, +1);
    for (int64_t i = 0; i < n * n; ++i) {
        double a = A[2 * i], b = A[2 * i + 1], cc = B[2 * i], d = B[2 * i + 1];
        A[2 * i] = a * cc - b * d;
        A[2 * i + 1] = a * d + b * cc;
    }
    fft_nd(A, N, -1);
    double scale = 1.0 / ((double)n * (double)n);
    for (int64_t kx = -c; kx <= c; ++kx)
        for (int64_t ky = 0; ky <= c; ++ky) {
            int64_t ix = (kx + n) % n, iy = ky;
            h[2 * ((kx + c) * K + ky)] = A[2 * (ix * n + iy)] * scale;
            h[2 * ((kx + c) * K + ky) + 1] = A[2 * (ix * n + iy) + 1] * scale;
        }
    free(A);
    free(B);
    return 0;
}

/* ------------------------------------------------ O7 MLP predictor (FP64) */

/* Network n_in -> H -> H -> H -> n_out with ReLU after the hidden layers;
 * parameters per layer W[i][o] (row-major) then b[o].  Loss: mean over the
 * n samples of softmax cross-entropy on outputs [0, n_q) with label yq and
 * on outputs [n_q, n_q + 2) with label yd (a label < 0 skips that term).
 * Writes the loss, the gradient of every parameter and the logits. */
HDCO_API int hdco_mlp_loss_grad(const double* P, int n_in, int H, int n_out, int n_q, const double* X,
                                const int* yq, const int* yd, int n, double* loss, double* grad,
                                double* logits)
{
    int dims[5] = { n_in, H, H, H, n_out };
    long off_w[4], off_b[4], np = 0;
    for (int l = 0; l < 4; ++l) {
        off_w[l] = np;
        np += (long)dims[l] * dims[l + 1];
        off_b[l] = np;
        np += dims[l + 1];
    }
    for (long k = 0; k < np; ++k) grad[k] = 0.0;
    double* z[5];
    double* a[5];
    double* dz[5];
    for (int l = 1; l <= 4; ++l) {
        z[l] = (double*)calloc((size_t)dims[l], sizeof(double));
        a[l] = (double*)calloc((size_t)dims[l], sizeof(double));
        dz[l] = (double*)calloc((size_t)dims[l], sizeof(double));
    }
    double total = 0.0;
    for (int s = 0; s < n; ++s) {
        /* forward */
        const double* in = X + (long)s * n_in;
        for (int l = 1; l <= 4; ++l) {
            const double* prev = (l == 1) ? in : a[l - 1];
            for (int o = 0; o < dims[l]; ++o) {
                double acc = P[off_b[l - 1] + o];
                for (int i = 0; i < dims[l - 1]; ++i) acc += prev[i] * P[off_w[l - 1] + (long)i * dims[l] + o];
                z[l][o] = acc;
                a[l][o] = (l < 4 && acc < 0.0) ? 0.0 : acc;
            }
        }
        for (int o = 0; o < n_out; ++o) {
            logits[(long)s * n_out + o] = z[4][o];
            dz[4][o] = 0.0;
        }
        /* two softmax cross-entropy heads */
        int lo[2] = { 0, n_q }, hi[2] = { n_q, n_q + 2 }, y[2] = { yq[s], yd[s] };
        for (int h = 0; h < 2; ++h) {
            if (y[h] < 0) continue;
            double mx = z[4][lo[h]];
            for (int k = lo[h]; k < hi[h]; ++k) mx = z[4][k] > mx ? z[4][k] : mx;
            double se = 0.0;
            for (int k = lo[h]; k < hi[h]; ++k) se += exp(z[4][k] - mx);
            double lse = mx + log(se);
            total += lse - z[4][lo[h] + y[h]];
            for (int k = lo[h]; k < hi[h]; ++k)
                dz[4][k] = (exp(z[4][k] - lse) - ((k - lo[h]) == y[h] ? 1.0 : 0.0)) / (double)n;
        }
        /* backward */
        for (int l = 4; l >= 1; --l) {
            const double* prev = (l == 1) ? in : a[l - 1];
            for (int o = 0; o < dims[l]; ++o) {
                grad[off_b[l - 1] + o] += dz[l][o];
                for (int i = 0; i < dims[l - 1]; ++i) grad[off_w[l - 1] + (long)i * dims[l] + o] += prev[i] * dz[l][o];
            }
            if (l > 1)
                for (int i = 0; i < dims[l - 1]; ++i) {
                    double acc = 0.0;
                    for (int o = 0; o < dims[l]; ++o) acc += dz[l][o] * P[off_w[l - 1] + (long)i * dims[l] + o];
                    dz[l - 1][i] = z[l - 1][i] > 0.0 ? acc : 0.0;
                }
        }
    }
    *loss = total / (double)n;
    for (int l = 1; l <= 4; ++l) { free(z[l]); free(a[l]); free(dz[l]); }
    return 0;
}

/* One Adam step (Kingma and Ba, 2015) with bias correction at step t >= 1. */
HDCO_API void hdco_adam_step(double* p, const double* g, double* m, double* v, long n, double lr, double b1,
                             double b2, double eps, long t)
{
    double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (long k = 0; k < n; ++k) {
        m[k] = b1 * m[k] + (1.0 - b1) * g[k];
        v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
        p[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

HDCO_API int hdco_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

HDCO_API void hdco_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

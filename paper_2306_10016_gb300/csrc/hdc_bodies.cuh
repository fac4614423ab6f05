// hdc_bodies.cuh -- block-level bodies of the residue kernels, shared by the
// one-pass kernels (hdc_kernels.cu) and the persistent batched kernel
// (hdc_batched.cu).  Every body is executed by all threads of a block,
// works in the shared memory it is given, and ends with a barrier so the
// block may run the next body on the same shared memory.
#pragma once

#include "hdc_fft.cuh"

namespace hdc {

// One residue r of one row: fold (Eq. 1 inner sum, then zeta_N^{r s}) of f
// and g, m-point forward FFTs, pointwise product (Section 2.4), inverse FFT
// (Eq. 2 inner sum); the unscaled result goes to hr[0..m).  smem: three
// swizzled buffers of m (3 smem_len(m) elements).  g has L valid elements,
// f has Lf <= L (zero beyond).  With p = q = 1 and Lf = L >= m the fold is a
// plain copy of the rows.
template <class V, bool R16 = false>
__device__ __forceinline__ void residue_row_body(const V* fr, const V* gr, V* hr, int64_t L, int64_t Lf, int m, int p,
                                                 int q, int r, const TwTab<V> twN, const V* __restrict__ twm,
                                                 const V* __restrict__ twml, const FftPlan& fp, V* smem, int tid,
                                                 int nthr)
{
    const int plen = (int)smem_len<V>(m);
    V* sa = smem;
    V* sb = sa + plen;
    V* sc = sb + plen;
    if (p == 1 && q == 1 && L >= m && Lf == L) {
#pragma unroll 4
        for (int s = tid; s < m; s += nthr) {
            sa[sidx<V, true>(s)] = fr[s];
            sb[sidx<V, true>(s)] = gr[s];
        }
    } else {
        for (int s = tid; s < m; s += nthr) {
            // block t = 0 carries zeta_q^0 = 1: no multiplication
            V af = s < Lf ? fr[s] : czero<V>(), ag = s < L ? gr[s] : czero<V>();
            for (int t = 1; t < p; ++t) {
                const int64_t j = (int64_t)t * m + s;
                if (j >= L) break;
                const V fv = j < Lf ? fr[j] : czero<V>(), gv = gr[j];
                if (r == 0) {
                    af = cadd(af, fv);
                    ag = cadd(ag, gv);
                } else {
                    const V w = twn(twN, rt_mod(r, t, q) * m);
                    af = cfma(fv, w, af);
                    ag = cfma(gv, w, ag);
                }
            }
            if (r != 0) {
                const V w = twn(twN, (int64_t)r * s);
                af = cmul(af, w);
                ag = cmul(ag, w);
            }
            sa[sidx<V, true>(s)] = af;
            sb[sidx<V, true>(s)] = ag;
        }
    }
    __syncthreads();
    if constexpr (sizeof(V) == 8) {
        // FP32, bound by shared-memory passes: each transform leaves its
        // result where its last stage wrote it, and the next one takes a
        // buffer that is free at that point as its scratch
        V* F = fft_smem_any<V, false, true, R16>(sa, sc, fp, 1, 1, m, twm, twml, tid, nthr);
        V* G = fft_smem_any<V, false, true, R16>(sb, F == sa ? sc : sa, fp, 1, 1, m, twm, twml, tid, nthr);
        for (int s = tid; s < m; s += nthr) F[sidx<V, true>(s)] = cmul(F[sidx<V, true>(s)], G[sidx<V, true>(s)]);
        __syncthreads();
        const V* H = fft_smem_any<V, true, true, R16>(F, G, fp, 1, 1, m, twm, twml, tid, nthr);
        for (int s = tid; s < m; s += nthr) hr[s] = H[sidx<V, true>(s)];
    } else {
        // FP64, bound by the FP64 pipe: most row plans up to 2048 points
        // have an even number of stages, and leaving the odd ones in place
        // measured no difference, so the results are copied back
        fft_smem<V, false, true, R16>(sa, sc, fp, 1, 1, m, twm, twml, tid, nthr);
        fft_smem<V, false, true, R16>(sb, sc, fp, 1, 1, m, twm, twml, tid, nthr);
        for (int s = tid; s < m; s += nthr) sa[sidx<V, true>(s)] = cmul(sa[sidx<V, true>(s)], sb[sidx<V, true>(s)]);
        __syncthreads();
        fft_smem<V, true, true, R16>(sa, sc, fp, 1, 1, m, twm, twml, tid, nthr);
        for (int s = tid; s < m; s += nthr) hr[s] = sa[sidx<V, true>(s)];
    }
    __syncthreads();
}

// Fold (Eq. 1 inner sum) of one input row x of L valid elements into the
// swizzled buffer dst: dst[s] = zeta_N^{r s} sum_{t < p} zeta_q^{r t} x[t m + s],
// s < m, with N = q m; no barrier.
template <class V>
__device__ __forceinline__ void fold_row(const V* x, int64_t L, int m, int p, int q, int r, const TwTab<V> twN,
                                         V* dst, int tid, int nthr)
{
    for (int s = tid; s < m; s += nthr) {
        V a = s < L ? x[s] : czero<V>(); // block t = 0: zeta_q^0 = 1
        for (int t = 1; t < p; ++t) {
            const int64_t j = (int64_t)t * m + s;
            if (j >= L) break;
            if (r == 0) a = cadd(a, x[j]);
            else a = cfma(x[j], twn(twN, rt_mod(r, t, q) * m), a);
        }
        if (r != 0) a = cmul(a, twn(twN, (int64_t)r * s));
        dst[sidx<V, true>(s)] = a;
    }
}

// Up to kMaxInputs input arrays of a multi-convolution (kernel argument).
template <class V> struct InPtrs {
    const V* x[kMaxInputs];
};

// Multi-convolution, one residue r of one row (offset boff into every
// input): fold (Eq. 1 inner sum) and m-point FFT of each of the nin inputs,
// then per DFT index either the product of all nin transforms (op 0, the
// nin-fold convolution) or the sum of the pairwise products
// F_0 F_1 + F_2 F_3 + ... (op 1, nin even); inverse FFT; the unscaled result
// goes to hr[0..m).  The sum accumulates in hr itself (each thread owns the
// same elements in every pass).  smem: three swizzled buffers of m.
template <class V>
__device__ __forceinline__ void residue_row_multi_body(const InPtrs<V>& in, int nin, int op, int64_t boff, V* hr,
                                                       int64_t L, int m, int p, int q, int r,
                                                       const TwTab<V> twN, const V* __restrict__ twm,
                                                       const V* __restrict__ twml, const FftPlan& fp, V* smem,
                                                       int tid, int nthr)
{
    const int plen = (int)smem_len<V>(m);
    V* sa = smem;
    V* sb = sa + plen;
    V* sc = sb + plen;
    for (int i = 0; i < nin; ++i) {
        // op 0: sa accumulates the product; op 1: sa holds F_{2j}, sb F_{2j+1}
        V* dst = (i == 0 || (op == 1 && (i & 1) == 0)) ? sa : sb;
        fold_row<V>(in.x[i] + boff, L, m, p, q, r, twN, dst, tid, nthr);
        __syncthreads();
        fft_smem<V, false, true>(dst, sc, fp, 1, 1, m, twm, twml, tid, nthr);
        if (op == 0 && i > 0) {
            for (int s = tid; s < m; s += nthr) sa[sidx<V, true>(s)] = cmul(sa[sidx<V, true>(s)], sb[sidx<V, true>(s)]);
            __syncthreads();
        } else if (op == 1 && (i & 1)) {
            for (int s = tid; s < m; s += nthr) {
                const V v = cmul(sa[sidx<V, true>(s)], sb[sidx<V, true>(s)]);
                hr[s] = (i == 1) ? v : cadd(hr[s], v);
            }
            __syncthreads();
        }
    }
    if (op == 1)
        for (int s = tid; s < m; s += nthr) sa[sidx<V, true>(s)] = hr[s];
    __syncthreads();
    fft_smem<V, true, true>(sa, sc, fp, 1, 1, m, twm, twml, tid, nthr);
    for (int s = tid; s < m; s += nthr) hr[s] = sa[sidx<V, true>(s)];
    __syncthreads();
}

// Unequal lengths with residue matching (Section 3.5, final algorithm for
// one dimension): g is transformed at mg = lam mf points with qg residues,
// f at mf points with qf = lam qg residues, both over the same N = qg mg.
// The DFT index qg lg + rg equals qf lf + rf for lg = lam lf + l, rf = qg l +
// rg, so residue rg of g pairs bin lam lf + l with bin lf of residue
// qg l + rg of f, l = 0 .. lam-1.  One block: fold g (residue rg), mg-point
// FFT; for each l: fold f (residue qg l + rg), mf-point FFT, multiply into
// the bins lam lf + l; inverse mg-point FFT; unscaled result to hr[0..mg).
// smem: three swizzled buffers of mg.
template <class V>
__device__ __forceinline__ void residue_row_lam_body(const V* fr, const V* gr, V* hr, int64_t Lf, int64_t Lg, int mf,
                                                     int mg, int lam, int pf, int pg, int qg, int rg,
                                                     const TwTab<V> twN, const V* __restrict__ twf,
                                                     const V* __restrict__ twfl, const FftPlan& fpf,
                                                     const V* __restrict__ twg, const V* __restrict__ twgl,
                                                     const FftPlan& fpg, V* smem, int tid, int nthr)
{
    const int plen = (int)smem_len<V>(mg);
    V* sa = smem;
    V* sb = sa + plen;
    V* sc = sb + plen;
    const int qf = qg * lam;
    fold_row<V>(gr, Lg, mg, pg, qg, rg, twN, sa, tid, nthr);
    __syncthreads();
    fft_smem<V, false, true>(sa, sc, fpg, 1, 1, mg, twg, twgl, tid, nthr);
    for (int l = 0; l < lam; ++l) {
        fold_row<V>(fr, Lf, mf, pf, qf, qg * l + rg, twN, sb, tid, nthr);
        __syncthreads();
        fft_smem<V, false, true>(sb, sc, fpf, 1, 1, mf, twf, twfl, tid, nthr);
        for (int lf = tid; lf < mf; lf += nthr) {
            const int k = sidx<V, true>(lf * lam + l);
            sa[k] = cmul(sa[k], sb[sidx<V, true>(lf)]);
        }
        __syncthreads();
    }
    fft_smem<V, true, true>(sa, sc, fpg, 1, 1, mg, twg, twgl, tid, nthr);
    for (int s = tid; s < mg; s += nthr) hr[s] = sa[sidx<V, true>(s)];
    __syncthreads();
}

// Real inputs (packed as z = f + i g): F and G at one DFT index from Z there
// (a) and Z at the mirrored index (b):  F = (a + conj b) / 2,
// G = (a - conj b) / (2 i);  returns their product H = F G.
template <class V> __device__ __forceinline__ V real_pair_product(V a, V b)
{
    using T = typename real_of<V>::type;
    const T h = (T)0.5;
    const V F = mkc<V>(h * (a.x + b.x), h * (a.y - b.y));
    const V G = mkc<V>(h * (a.y + b.y), -h * (a.x - b.x));
    return cmul(F, G);
}

// One kept residue r (2 r <= q) of one packed real row z: fold and m-point FFT
// of residue r and of its conjugate partner r' = (q - r) mod q, F and G from
// the pair (bin l of r against bin (m - l) mod m of r' = 0 when r = 0, bin
// m - 1 - l of r' otherwise), H = F G, inverse FFT; the unscaled result goes
// to hr[0..m).  smem: three swizzled buffers of m.
template <class V>
__device__ __forceinline__ void residue_row_real_body(const V* zr, V* hr, int64_t L, int m, int p, int q, int r,
                                                      const TwTab<V> twN, const V* __restrict__ twm,
                                                      const V* __restrict__ twml, const FftPlan& fp, V* smem, int tid,
                                                      int nthr)
{
    const int plen = (int)smem_len<V>(m);
    V* sa = smem;
    V* sb = sa + plen;
    V* sc = sb + plen;
    const int rp = (q - r) % q;
    fold_row<V>(zr, L, m, p, q, r, twN, sa, tid, nthr);
    __syncthreads();
    fft_smem<V, false, true>(sa, sc, fp, 1, 1, m, twm, twml, tid, nthr);
    V* pb = sa;
    if (rp != r) {
        fold_row<V>(zr, L, m, p, q, rp, twN, sb, tid, nthr);
        __syncthreads();
        fft_smem<V, false, true>(sb, sc, fp, 1, 1, m, twm, twml, tid, nthr);
        pb = sb;
    }
    for (int l = tid; l < m; l += nthr) {
        const int lp = r == 0 ? (m - l) % m : m - 1 - l;
        sc[sidx<V, true>(l)] = real_pair_product(sa[sidx<V, true>(l)], pb[sidx<V, true>(lp)]);
    }
    __syncthreads();
    fft_smem<V, true, true>(sc, sa, fp, 1, 1, m, twm, twml, tid, nthr);
    for (int s = tid; s < m; s += nthr) hr[s] = sc[sidx<V, true>(s)];
    __syncthreads();
}

// Split route, real inputs: row l1 of kept residue r (ya, after the column
// pass) against row l1' of its partner (yb): m2-point FFTs of both, H = F G
// per bin (bin l2 against (m2 - l2) mod m2 when r = 0 and l1 = 0, else
// m2 - 1 - l2), inverse FFT into yh.  smem: three swizzled buffers of m2.
template <class V>
__device__ __forceinline__ void rows_real_pair_body(const V* ya, const V* yb, V* yh, int m2, int r, int l1,
                                                    const V* __restrict__ twm, const V* __restrict__ twml,
                                                    const FftPlan& fp, V* smem, int tid, int nthr)
{
    const int plen = (int)smem_len<V>(m2);
    V* sa = smem;
    V* sb = sa + plen;
    V* sc = sb + plen;
    for (int s = tid; s < m2; s += nthr) {
        sa[sidx<V, true>(s)] = ya[s];
        sb[sidx<V, true>(s)] = yb[s];
    }
    __syncthreads();
    fft_smem<V, false, true>(sa, sc, fp, 1, 1, m2, twm, twml, tid, nthr);
    fft_smem<V, false, true>(sb, sc, fp, 1, 1, m2, twm, twml, tid, nthr);
    const bool wrap = r == 0 && l1 == 0;
    for (int l = tid; l < m2; l += nthr) {
        const int lp = wrap ? (m2 - l) % m2 : m2 - 1 - l;
        sc[sidx<V, true>(l)] = real_pair_product(sa[sidx<V, true>(l)], sb[sidx<V, true>(lp)]);
    }
    __syncthreads();
    fft_smem<V, true, true>(sc, sa, fp, 1, 1, m2, twm, twml, tid, nthr);
    for (int s = tid; s < m2; s += nthr) yh[s] = sc[sidx<V, true>(s)];
    __syncthreads();
}

// Loads a thread of a column-tile body keeps in flight at a time: an FP32
// tile needs more of them to cover the memory latency.
template <class V> constexpr int kColLoads = sizeof(V) == 8 ? 8 : 4;

// Second half of the strided fold + FFT pass: the folded tile (ma x C,
// element i C + cl) is in buf and the block is synchronised; FFT of size ma
// over the tile's columns, then column c0 + cl (< Cn) of row l goes to
// yb[l ystride + c], times zeta_{Nf/q}^{l c} if post: in FP64 from tpm[c ma + l]
// when the caller has that column-major table (Nf/q = ma Cn), else from twNf.
template <class V, bool R16 = false>
__device__ __forceinline__ void fft_cols_store_body(V* buf, V* tmp, V* yb, int64_t Cn, int ma, int q, int64_t c0,
                                                    int C, int post, int64_t ystride, const TwTab<V> twNf,
                                                    const V* __restrict__ tpm,
                                                    const V* __restrict__ twma, const V* __restrict__ twmal,
                                                    const FftPlan& fp, int tid, int nthr)
{
    const V* res = buf;
    if (ma > 1) res = fft_smem_any<V, false, false, R16>(buf, tmp, fp, C, C, 1, twma, twmal, tid, nthr);
    for (int e = tid; e < ma * C; e += nthr) {
        const int l = div_idx(e, C), cl = e - l * C;
        const int64_t c = c0 + cl;
        if (c >= Cn) continue;
        V v = res[e];
        if (post && l != 0 && c != 0) v = cmul(v, (sizeof(V) == 16 && tpm) ? __ldg(tpm + c * ma + l) : twn(twNf, (int64_t)l * c * q));
        yb[(int64_t)l * ystride + c] = v;
    }
    __syncthreads();
}

// Fold along a strided axis and FFT of size ma over it, for the columns
// c0 .. c0+C-1 (< Cn) of one input x (view x[a][c], a = t ma + i, element
// valid iff a Cn + c < Lvalid); residue r; result to yb[l ystride + c],
// times zeta_{Nf/q}^{l c} if post.  smem: 2 smem_len(ma C).
template <class V, bool R16 = false>
__device__ __forceinline__ void fold_fft_cols_body(const V* x, V* yb, int64_t Cn, int ma, int p, int q, int64_t Nf,
                                                   int64_t cs, int64_t cc, int64_t Lvalid, int r, int64_t c0, int C,
                                                   int post, int64_t ystride, const TwTab<V> twNf,
                                                   const V* __restrict__ tpm,
                                                   const V* __restrict__ twma, const V* __restrict__ twmal,
                                                   const FftPlan& fp, V* smem, int tid, int nthr)
{
    V* buf = smem;
    V* tmp = buf + smem_len<V>(ma * C);
    const int64_t mq = Nf / q;
    // four elements per thread at a time, so their loads are in flight
    // together (in FP32 also two fold blocks of each: the FP32 pass is bound
    // by memory latency, the FP64 one by its arithmetic, which this would
    // slow); element e = i C + cl of the tile is column c0 + cl, row i
    constexpr int U = 4;
    const int n = ma * C;
    for (int e0 = tid; e0 < n; e0 += U * nthr) {
        V acc[U];
        int64_t base[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nthr;
            const int i = div_idx(e, C), cl = e - i * C;
            const int64_t c = c0 + cl;
            base[u] = (e < n && c < Cn) ? (int64_t)i * Cn + c : -1;
        }
        if constexpr (sizeof(V) == 8) {
            for (int t = 0; t < p; t += 2) {
                const int64_t off = (int64_t)t * ma * Cn, off2 = off + (int64_t)ma * Cn;
                V xa[U], xb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    xa[u] = (base[u] >= 0 && base[u] + off < Lvalid) ? x[base[u] + off] : czero<V>();
                    xb[u] = (t + 1 < p && base[u] >= 0 && base[u] + off2 < Lvalid) ? x[base[u] + off2] : czero<V>();
                }
                // block t = 0 carries zeta_q^0 = 1: no multiplication
                const V wa = (r == 0 || t == 0) ? czero<V>() : twn(twNf, rt_mod(r, t, q) * mq);
                const V wb = r == 0 ? czero<V>() : twn(twNf, rt_mod(r, (t + 1), q) * mq);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (t == 0) acc[u] = xa[u];
                    else acc[u] = r == 0 ? cadd(acc[u], xa[u]) : cfma(xa[u], wa, acc[u]);
                    if (t + 1 < p) acc[u] = r == 0 ? cadd(acc[u], xb[u]) : cfma(xb[u], wb, acc[u]);
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u)
                // block t = 0 carries zeta_q^0 = 1: no multiplication
                acc[u] = (base[u] >= 0 && base[u] < Lvalid) ? x[base[u]] : czero<V>();
            for (int t = 1; t < p; ++t) {
                const int64_t off = (int64_t)t * ma * Cn;
                if (off >= Lvalid) break;
                const V w = r == 0 ? czero<V>() : twn(twNf, rt_mod(r, t, q) * mq);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (base[u] < 0 || base[u] + off >= Lvalid) continue;
                    const V xv = x[base[u] + off];
                    acc[u] = r == 0 ? cadd(acc[u], xv) : cfma(xv, w, acc[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nthr;
            if (e >= n) break;
            V a = acc[u];
            if (r != 0 && base[u] >= 0) {
                const int i = div_idx(e, C), cl = e - i * C;
                a = cmul(a, twn(twNf, (int64_t)r * (i * cs + (c0 + cl) * cc)));
            }
            buf[e] = a;
        }
    }
    __syncthreads();
    fft_cols_store_body<V, R16>(buf, tmp, yb, Cn, ma, q, c0, C, post, ystride, twNf, tpm, twma, twmal, fp, tid, nthr);
}

// Inverse FFT of size ma along the strided axis of yb[l][c] (row length Cn)
// for columns c0 .. c0+C-1, in place, after multiplying by
// conj(zeta_{Nf/q}^{l c}) if pre.  smem: 2 smem_len(ma C).
template <class V, bool R16 = false>
__device__ __forceinline__ void ifft_cols_body(V* yb, int64_t Cn, int ma, int q, int64_t Nf, int64_t c0, int C,
                                               int pre, const TwTab<V> twNf, const V* __restrict__ tpm,
                                               const V* __restrict__ twma,
                                               const V* __restrict__ twmal, const FftPlan& fp, V* smem, int tid,
                                               int nthr)
{
    V* buf = smem;
    V* tmp = buf + smem_len<V>(ma * C);
    // U elements per thread at a time, so their loads are in flight together
    constexpr int U = kColLoads<V>;
    const int n = ma * C;
    for (int e0 = tid; e0 < n; e0 += U * nthr) {
        V v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nthr;
            const int l = div_idx(e, C), cl = e - l * C;
            const int64_t c = c0 + cl;
            v[u] = (e < n && c < Cn) ? yb[(int64_t)l * Cn + c] : czero<V>();
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + u * nthr;
            if (e >= n) break;
            const int l = div_idx(e, C), cl = e - l * C;
            const int64_t c = c0 + cl;
            if (pre && l != 0 && c != 0 && c < Cn)
                    v[u] = cmulc(v[u], (sizeof(V) == 16 && tpm) ? __ldg(tpm + c * ma + l) : twn(twNf, (int64_t)l * c * q));
            buf[e] = v[u];
        }
    }
    __syncthreads();
    const V* res = buf;
    if (ma > 1) res = fft_smem_any<V, true, false, R16>(buf, tmp, fp, C, C, 1, twma, twmal, tid, nthr);
    for (int e = tid; e < ma * C; e += nthr) {
        const int s = div_idx(e, C), cl = e - s * C;
        const int64_t c = c0 + cl;
        if (c < Cn) yb[(int64_t)s * Cn + c] = res[e];
    }
    __syncthreads();
}

// Inverse FFT of size ma along the strided axis and unfold, fused: for the
// columns c0 .. c0+C-1 of one row, residues r = r0 + rr (rr < Dg) in order:
// load y_rr = y + rr * rstride (times conj(zeta_{Nf/q}^{l c}) if pre),
// inverse FFT, then add conj(zeta_Nf^{r (i cs + c cc)}) conj(zeta_q^{r t})
// h[i][c] to the output at lin = (t ma + i) Cn + c, t < p, lo <= lin < hi,
// stored at ob[lin - lo]: these outputs belong to this tile alone.  The
// first residue of the first pass writes instead of adding; the last of the
// last pass scales.  smem: 2 smem_len(ma C).
template <class V, bool R16 = false>
__device__ __forceinline__ void ifft_unfold_cols_body(const V* y, int64_t rstride, V* ob, int64_t Cn, int ma, int p,
                                                      int q, int64_t Nf, int64_t cs, int64_t cc, int64_t lo,
                                                      int64_t hi, int r0, int Dg, int first, int last,
                                                      typename real_of<V>::type scale, int64_t c0, int C, int pre,
                                                      const TwTab<V> twNf, const V* __restrict__ tpm,
                                                      const V* __restrict__ twma,
                                                      const V* __restrict__ twmal, const FftPlan& fp, V* smem,
                                                      int tid, int nthr)
{
    V* buf = smem;
    V* tmp = buf + smem_len<V>(ma * C);
    const int64_t mq = Nf / q;
    constexpr int U = kColLoads<V>;
    const int n = ma * C;
    for (int rr = 0; rr < Dg; ++rr) {
        const int r = r0 + rr;
        const V* yb = y + (int64_t)rr * rstride;
        for (int e0 = tid; e0 < n; e0 += U * nthr) {
            V v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * nthr;
                const int l = div_idx(e, C), cl = e - l * C;
                const int64_t c = c0 + cl;
                v[u] = (e < n && c < Cn) ? yb[(int64_t)l * Cn + c] : czero<V>();
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * nthr;
                if (e >= n) break;
                const int l = div_idx(e, C), cl = e - l * C;
                const int64_t c = c0 + cl;
                if (pre && l != 0 && c != 0 && c < Cn)
                    v[u] = cmulc(v[u], (sizeof(V) == 16 && tpm) ? __ldg(tpm + c * ma + l) : twn(twNf, (int64_t)l * c * q));
                buf[e] = v[u];
            }
        }
        __syncthreads();
        const V* res = buf;
        if (ma > 1) res = fft_smem_any<V, true, false, R16>(buf, tmp, fp, C, C, 1, twma, twmal, tid, nthr);
        const bool init = first && rr == 0, fin = last && rr == Dg - 1;
        for (int e = tid; e < n; e += nthr) {
            const int i = div_idx(e, C), cl = e - i * C;
            const int64_t c = c0 + cl;
            if (c >= Cn) continue;
            V hv = res[e];
            if (r != 0) hv = cmulc(hv, twn(twNf, (int64_t)r * (i * cs + c * cc)));
            for (int t = 0; t < p; ++t) {
                const int64_t lin = ((int64_t)t * ma + i) * Cn + c;
                if (lin >= hi) break;
                if (lin < lo) continue;
                V v = (r != 0 && t != 0) ? cmulc(hv, twn(twNf, rt_mod(r, t, q) * mq)) : hv;
                if (!init) v = cadd(ob[lin - lo], v);
                if (fin) v = cscale(v, scale);
                ob[lin - lo] = v;
            }
        }
        __syncthreads();
    }
}

// Unfold of one element (i, c) of one row: the output at linear index
// lin = (t ma + i) Cn + c, for every t < p with lo <= lin < hi, is
// sum_{rr < Dg} conj(zeta_Nf^{r (i cs + c cc)}) conj(zeta_q^{r t}) h_rr[i][c]
// (h_rr = h + rr * hstride, residues r = r0 + rr in increasing order),
// written to ob[lin - lo]; added to the previous contents unless first,
// scaled if last.  PT outputs are accumulated per sweep over the residues.
template <class V, int PT>
__device__ __forceinline__ void unfold_elem(V* ob, const V* __restrict__ h, int64_t hstride, int64_t Cn,
                                            int64_t ma, int64_t i, int64_t c, int p, int q, int64_t Nf, int64_t cs,
                                            int64_t cc, int64_t lo, int64_t hi, int r0, int Dg, int first, int last,
                                            typename real_of<V>::type scale, const TwTab<V> twNf)
{
    const int64_t mq = Nf / q;
    for (int t0 = 0; t0 < p; t0 += PT) {
        if ((((int64_t)t0 * ma + i) * Cn + c) >= hi) break;
        const int tl = (t0 + PT - 1 < p) ? t0 + PT - 1 : p - 1;
        if ((((int64_t)tl * ma + i) * Cn + c) < lo) continue;
        V acc[PT];
#pragma unroll
        for (int tt = 0; tt < PT; ++tt) acc[tt] = czero<V>();
        // FP32: the residues' values are loaded four at a time before they
        // are used, so their loads are in flight together (FP64, bound by
        // its arithmetic, measured 1-3 % slower that way)
        constexpr int RB = sizeof(V) == 8 ? 4 : 1;
        for (int rb = 0; rb < Dg; rb += RB) {
            V hb[RB];
#pragma unroll
            for (int k = 0; k < RB; ++k)
                hb[k] = rb + k < Dg ? h[(int64_t)(rb + k) * hstride + i * Cn + c] : czero<V>();
#pragma unroll
            for (int k = 0; k < RB; ++k) {
                if (rb + k >= Dg) break;
                const int r = r0 + rb + k;
                V hv = hb[k];
                if (r != 0) hv = cmulc(hv, twn(twNf, (int64_t)r * (i * cs + c * cc)));
#pragma unroll
                for (int tt = 0; tt < PT; ++tt) {
                    const int t = t0 + tt;
                    if (t < p) {
                        if (r == 0 || t == 0) acc[tt] = cadd(acc[tt], hv);
                        else acc[tt] = cfmac(hv, twn(twNf, rt_mod(r, t, q) * mq), acc[tt]);
                    }
                }
            }
        }
#pragma unroll
        for (int tt = 0; tt < PT; ++tt) {
            const int t = t0 + tt;
            if (t >= p) break;
            const int64_t lin = ((int64_t)t * ma + i) * Cn + c;
            if (lin >= hi) break;
            if (lin < lo) continue;
            V v = acc[tt];
            if (!first) v = cadd(v, ob[lin - lo]);
            if (last) v = cscale(v, scale);
            ob[lin - lo] = v;
        }
    }
}

} // namespace hdc

// hdc_hermitian.cu -- the inner (half-stored) axis of the centered Hermitian
// 2-D convolution, on half the data and half the transforms of the complex
// route.
//
// The inputs are the ky >= 0 halves of two spectra with f(-k) = conj f(k)
// on the box |kx|, |ky| <= c (c = K - 1); the convolution h = f * g on the
// box is the spectrum of the product of the two real fields u, v whose
// spectra f and g are (the dealiased pseudo-spectral product, padded by the
// 3/2 rule: N >= 3c + 1 per axis).  After the residue transform of the
// outer axis (kx, index a = kx + c; the kernels of the N-D route on the K
// half columns only), each transformed row at outer bin x holds
// F_s(x, ky) = zeta_Nx^{c x} F_x(ky) for ky >= 0, where F_x is Hermitian in
// ky; the other half is F_s(x, -ky) = zeta_Nx^{2 c x} conj F_s(x, ky).  Along
// ky (index j = ky + c) one block takes two rows x1, x2 and, for every
// residue r of the ky axis (Eq. 1, Eq. 2):
//  - folds and transforms the packed row z = F_s + i G_s of each (the half
//    it does not store comes from the mirror rule above), so one transform
//    gives both fields: zeta^{-c x - c y} Z(y) = u(x, y) + i v(x, y);
//  - forms the real product w = u v of each row and packs the pair,
//    Q(y) = zeta_Ny^{2 c y} (w1 + i w2);
//  - inverse-transforms Q and unfolds it into the outputs n = ky + 2c,
//    ky in [-c, c], accumulated on chip over the residues;
// then splits the pair by Hermitian symmetry (the output of a real w is
// Hermitian: h1 = (q(2c+k) + conj q(2c-k)) / 2, h2 = (q(2c+k) - conj q(2c-k)) / 2i)
// and writes each row's k >= 0 half times zeta_Nx^{2 c x}, the value the
// outer axis' inverse transform and unfold expect.  Per pair of rows and
// residue: two forward and one inverse transform instead of six.
#include <cuda_runtime.h>

#include <stdint.h>

#include "hdc.h"
#include "hdc_fft.cuh"
#include "hdc_internal.h"

namespace hdc {

template <class V> struct HermRowsArgs {
    const V* wf;      // rows of F_s, K values each
    const V* wg;      // rows of G_s
    V* wh;            // output rows, K values each
    int64_t B;        // problems per outer-residue block
    int64_t mx;       // rows per (outer residue, problem) block
    int K, my, qy, qx;
    int64_t Nx, Ny;
    int r0;           // first outer residue of the pass
    typename real_of<V>::type scale; // 1 / Ny
    TwTab<V> twNx, twNy;
    const V* twm;
    const V* twml;
    FftPlan fp;
};

// f + i g
template <class V> __device__ __forceinline__ V pack_fg(V f, V g) { return mkc<V>(f.x - g.y, f.y + g.x); }

// The packed row z = F_s + i G_s of outer bin x at ky in [-c, c], times
// zeta_Nx^{-c x} (= conj sx): stored for ky >= 0; for ky < 0 the mirror
// rule gives conj z(-ky) zeta_Nx^{2 c x} zeta_Nx^{-c x} = conj z(-ky) sx.
template <class V>
__device__ __forceinline__ V herm_z(const V* F, const V* G, int64_t ky, V sx)
{
    if (ky >= 0) return cmulc(pack_fg(F[ky], G[ky]), sx);
    const V f = F[-ky], g = G[-ky];
    return cmul(pack_fg(mkc<V>(f.x, -f.y), mkc<V>(g.x, -g.y)), sx);
}

// Shared memory: Z, the two packed rows side by side (element s of row t at
// 2 s + t), a scratch half T of the same size (the transforms of both rows
// run as one two-column transform), and, with several ky residues, the
// 2c + 1 output accumulators.
//
// Both ky sequences are laid out cyclically (ky at ky mod Ny), so the
// forward transform of z times zeta_Nx^{-c x} is u + i v directly and the
// inverse transform of w1 + i w2 holds the outputs ky at ky mod Ny: the
// phases zeta^{-c y} and zeta^{2 c y} of the window frame become index
// shifts (a product by zeta_N^{a y} on the bins is a cyclic shift by a).
template <class V>
__global__ void __launch_bounds__(kMaxThreads) k_hermitian_rows(const __grid_constant__ HermRowsArgs<V> a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    using T = typename real_of<V>::type;
    const int64_t npair = (a.mx + 1) / 2;
    const int64_t blk = blockIdx.x / npair;           // (outer residue rr, problem b)
    const int64_t l1 = 2 * (blockIdx.x - blk * npair); // first row of the pair
    const bool two = l1 + 1 < a.mx;
    const int rr = (int)(blk / a.B);
    const int rx = a.r0 + rr;
    const int c = a.K - 1, my = a.my, qy = a.qy;
    const int64_t Ny = a.Ny;
    const int zlen = (int)smem_len<V>(2 * my);
    V* Z = reinterpret_cast<V*>(smraw);
    V* Tm = Z + zlen;
    V* acc = Tm + zlen;                               // ky + c, ky in [-c, c] (qy > 1)
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int64_t row1 = blk * a.mx + l1;
    const V* F1 = a.wf + row1 * a.K;
    const V* G1 = a.wg + row1 * a.K;
    const V* F2 = F1 + a.K;
    const V* G2 = G1 + a.K;
    // outer bins x = qx l + rx of the two rows and their phases
    const int64_t x1 = (int64_t)a.qx * l1 + rx, x2 = x1 + a.qx;
    const V e1 = twn(a.twNx, (2 * (int64_t)c * x1) % a.Nx), e2 = twn(a.twNx, (2 * (int64_t)c * x2) % a.Nx);
    const V s1 = twn(a.twNx, ((int64_t)c * x1) % a.Nx), s2 = twn(a.twNx, ((int64_t)c * x2) % a.Nx);
    if (qy > 1)
        for (int e = tid; e < 2 * c + 1; e += nthr) acc[e] = czero<V>();
    const V* Qr = nullptr;
    for (int r = 0; r < qy; ++r) {
        // fold (Eq. 1 inner sum, then zeta_Ny^{r s}) of both packed rows:
        // element (s, t) of the two-column tile, thread e on row t = e & 1
        for (int e = tid; e < 2 * my; e += nthr) {
            const int s = e >> 1, t1 = e & 1;
            const V* F = t1 ? F2 : F1;
            const V* G = t1 ? G2 : G1;
            const V sx = t1 ? s2 : s1;
            V v = czero<V>();
            if (!t1 || two) {
                for (int t = 0; t < qy; ++t) {
                    const int64_t i = (int64_t)t * my + s;
                    int64_t ky;
                    if (i <= c) ky = i;
                    else if (i >= Ny - c) ky = i - Ny;
                    else continue;
                    const V z = herm_z(F, G, ky, sx);
                    v = (r == 0 || t == 0) ? cadd(v, z) : cfma(z, twn(a.twNy, rt_mod(r, t, qy) * my), v);
                }
                if (r != 0) v = cmul(v, twn(a.twNy, (int64_t)r * s));
            }
            Z[sidx<V, true>(e)] = v;
        }
        __syncthreads();
        // both rows' my-point transforms at once (two columns): bins
        // y = qy l + r of u + i v per row; the real products, packed
        fft_smem<V, false, true>(Z, Tm, a.fp, 2, 2, 1, a.twm, a.twml, tid, nthr);
        for (int l = tid; l < my; l += nthr) {
            const V uv1 = Z[sidx<V, true>(2 * l)], uv2 = Z[sidx<V, true>(2 * l + 1)];
            Tm[sidx<V, true>(l)] = mkc<V>(uv1.x * uv1.y, uv2.x * uv2.y);
        }
        __syncthreads();
        Qr = fft_smem_any<V, true, true>(Tm, Z, a.fp, 1, 1, my, a.twm, a.twml, tid, nthr);
        if (qy == 1) break;                           // the outputs stay in Qr
        // unfold (Eq. 2 outer sums): output ky at cyclic index i = ky mod Ny
        for (int s = tid; s < my; s += nthr) {
            V hv = Qr[sidx<V, true>(s)];
            if (r != 0) hv = cmulc(hv, twn(a.twNy, (int64_t)r * s));
            for (int t = 0; t < qy; ++t) {
                const int64_t i = (int64_t)t * my + s;
                int64_t ky;
                if (i <= c) ky = i;
                else if (i >= Ny - c) ky = i - Ny;
                else continue;
                const V v = (r != 0 && t != 0) ? cmulc(hv, twn(a.twNy, rt_mod(r, t, qy) * my)) : hv;
                acc[ky + c] = cadd(acc[ky + c], v);
            }
        }
        __syncthreads();
    }
    // split the pair (each row's output is Hermitian in ky) and write the
    // k >= 0 halves, scaled by 1 / Ny and times zeta_Nx^{2 c x}
    V* H1 = a.wh + row1 * a.K;
    for (int k = tid; k <= c; k += nthr) {
        V A, Bm;
        if (qy == 1) {
            A = Qr[sidx<V, true>(k)];
            Bm = Qr[sidx<V, true>(k == 0 ? 0 : my - k)];
        } else {
            A = acc[c + k];
            Bm = acc[c - k];
        }
        const T h = (T)0.5 * a.scale;
        const V h1 = mkc<V>(h * (A.x + Bm.x), h * (A.y - Bm.y));
        H1[k] = cmul(h1, e1);
        if (two) {
            // (A - conj Bm) / (2i)
            const V h2 = mkc<V>(h * (A.y + Bm.y), -h * (A.x - Bm.x));
            H1[a.K + k] = cmul(h2, e2);
        }
    }
}

template <typename T>
cudaError_t launch_hermitian_rows(const cx<T>* wf, const cx<T>* wg, cx<T>* wh, int64_t nblk, int64_t B, int64_t mx,
                                  int64_t K, int64_t my, int64_t qy, int64_t Nx, int64_t qx, int64_t r0,
                                  cudaStream_t st)
{
    using V = cx<T>;
    if (nblk <= 0 || mx <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    HermRowsArgs<V> a;
    a.twNx = tw_table<T>(Nx, &e);
    if (e != cudaSuccess) return e;
    a.twNy = tw_table<T>(qy * my, &e);
    if (e != cudaSuccess) return e;
    a.twm = twiddles_fft<T>(my, false, &e);
    if (e != cudaSuccess) return e;
    a.twml = twiddles_fft<T>(my, true, &e);
    if (e != cudaSuccess) return e;
    a.fp = fft_plan<T>(my);
    a.wf = wf;
    a.wg = wg;
    a.wh = wh;
    a.B = B;
    a.mx = mx;
    a.K = (int)K;
    a.my = (int)my;
    a.qy = (int)qy;
    a.qx = (int)qx;
    a.Nx = Nx;
    a.Ny = qy * my;
    a.r0 = (int)r0;
    a.scale = (T)(1.0 / (double)(qy * my));
    // one thread per radix-8 butterfly of the two-column transform
    int thr = (int)((2 * my / 8 + 31) / 32 * 32);
    thr = thr < 64 ? 64 : (thr > kMaxThreads ? kMaxThreads : thr);
    const size_t smem = (size_t)(2 * smem_len<V>(2 * my) + (qy > 1 ? 2 * K - 1 : 0)) * sizeof(V);
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_hermitian_rows<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return e;
    if (preparing()) return cudaSuccess;
    const int64_t npair = (mx + 1) / 2;
    const double n_in = 2.0 * K - 1.0;
    // model: per pair of rows and residue two forward and one inverse
    // my-point FFT, the folds of both packed rows (8 flops per element),
    // the products and the unfold
    LaunchScope ls(K_HERMITIAN_ROWS, st,
                   (double)(nblk * npair) * qy * (3.0 * fft_flops((double)my) + 16.0 * n_in + 20.0 * my + 8.0 * n_in),
                   (double)(nblk * mx) * 3.0 * K * sizeof(V));
    k_hermitian_rows<V><<<(unsigned)(nblk * npair), thr, smem, st>>>(a);
    return cudaGetLastError();
}
template cudaError_t launch_hermitian_rows<double>(const cx<double>*, const cx<double>*, cx<double>*, int64_t, int64_t,
                                                   int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,
                                                   cudaStream_t);
template cudaError_t launch_hermitian_rows<float>(const cx<float>*, const cx<float>*, cx<float>*, int64_t, int64_t,
                                                  int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,
                                                  cudaStream_t);

} // namespace hdc

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
    int K, my, py, qy, qx, pout; // pout = ceil((3c + 1) / my) output blocks
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

// Element j (< 2c + 1) of the packed row z = F_s + i G_s of outer bin x:
// stored for j >= c, mirrored with e = zeta_Nx^{2 c x} below.
template <class V>
__device__ __forceinline__ V herm_z(const V* F, const V* G, int64_t j, int c, V e)
{
    if (j >= c) return pack_fg(F[j - c], G[j - c]);
    const V f = F[c - j], g = G[c - j];
    return cmul(pack_fg(mkc<V>(f.x, -f.y), mkc<V>(g.x, -g.y)), e);
}

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
    const int plen = (int)smem_len<V>(my);
    V* z1 = reinterpret_cast<V*>(smraw);
    V* z2 = z1 + plen;
    V* tmp = z2 + plen;
    V* acc = tmp + plen;                              // outputs n = c .. 3c
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
    const int64_t n_in = 2 * (int64_t)c + 1;
    for (int e = tid; e < 2 * c + 1; e += nthr) acc[e] = czero<V>();
    for (int r = 0; r < qy; ++r) {
        // fold (Eq. 1 inner sum, then zeta_Ny^{r s}) of both packed rows
        for (int s = tid; s < my; s += nthr) {
            V a1 = s < n_in ? herm_z(F1, G1, s, c, e1) : czero<V>();
            V a2 = (two && s < n_in) ? herm_z(F2, G2, s, c, e2) : czero<V>();
            for (int t = 1; t < a.py; ++t) {
                const int64_t j = (int64_t)t * my + s;
                if (j >= n_in) break;
                const V w = twn(a.twNy, (((int64_t)r * t) % qy) * my);
                a1 = cfma(herm_z(F1, G1, j, c, e1), w, a1);
                if (two) a2 = cfma(herm_z(F2, G2, j, c, e2), w, a2);
            }
            if (r != 0) {
                const V w = twn(a.twNy, (int64_t)r * s);
                a1 = cmul(a1, w);
                a2 = cmul(a2, w);
            }
            z1[sidx<V, true>(s)] = a1;
            z2[sidx<V, true>(s)] = a2;
        }
        __syncthreads();
        fft_smem<V, false, true>(z1, tmp, a.fp, 1, 1, my, a.twm, a.twml, tid, nthr);
        fft_smem<V, false, true>(z2, tmp, a.fp, 1, 1, my, a.twm, a.twml, tid, nthr);
        // bins y = qy l + r: the fields u + i v of each row, their real
        // products, packed and shifted back to the window's frame
        for (int l = tid; l < my; l += nthr) {
            const int64_t y = (int64_t)qy * l + r;
            const V py = twn(a.twNy, ((int64_t)c * y) % a.Ny);
            const V p2 = twn(a.twNy, (2 * (int64_t)c * y) % a.Ny);
            const int k = sidx<V, true>(l);
            const V uv1 = cmulc(cmulc(z1[k], s1), py);
            const V uv2 = cmulc(cmulc(z2[k], s2), py);
            const T w1 = uv1.x * uv1.y, w2 = uv2.x * uv2.y;
            z1[k] = cmul(mkc<V>(w1, w2), p2);
        }
        __syncthreads();
        fft_smem<V, true, true>(z1, tmp, a.fp, 1, 1, my, a.twm, a.twml, tid, nthr);
        // unfold (Eq. 2 outer sums) into the outputs n in [c, 3c]
        for (int s = tid; s < my; s += nthr) {
            V hv = z1[sidx<V, true>(s)];
            if (r != 0) hv = cmulc(hv, twn(a.twNy, (int64_t)r * s));
            for (int t = 0; t < a.pout; ++t) {
                const int64_t n = (int64_t)t * my + s;
                if (n > 3 * (int64_t)c) break;
                if (n < c) continue;
                const V v = (r != 0 && t != 0) ? cmulc(hv, twn(a.twNy, (((int64_t)r * t) % qy) * my)) : hv;
                acc[n - c] = cadd(acc[n - c], v);
            }
        }
        __syncthreads();
    }
    // split the pair (each row's output is Hermitian in ky) and write the
    // k >= 0 halves, scaled by 1 / Ny and times zeta_Nx^{2 c x}
    V* H1 = a.wh + row1 * a.K;
    for (int k = tid; k <= c; k += nthr) {
        const V A = acc[c + k], Bm = acc[c - k];
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
                                  int64_t K, int64_t my, int64_t py, int64_t qy, int64_t Nx, int64_t qx, int64_t r0,
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
    a.py = (int)py;
    a.qy = (int)qy;
    a.qx = (int)qx;
    a.pout = (int)((3 * (K - 1) + 1 + my - 1) / my);
    a.Nx = Nx;
    a.Ny = qy * my;
    a.r0 = (int)r0;
    a.scale = (T)(1.0 / (double)(qy * my));
    int thr = (int)((my / 8 + 31) / 32 * 32);
    thr = thr < 64 ? 64 : (thr > kMaxThreads ? kMaxThreads : thr);
    const size_t smem = (size_t)(3 * smem_len<V>(my) + 2 * K - 1) * sizeof(V);
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
                                                   int64_t, cudaStream_t);
template cudaError_t launch_hermitian_rows<float>(const cx<float>*, const cx<float>*, cx<float>*, int64_t, int64_t,
                                                  int64_t, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t,
                                                  int64_t, cudaStream_t);

} // namespace hdc

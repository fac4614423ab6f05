// hdc_internal.h -- host-side declarations shared by the translation units of
// the library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "hdc_fft.cuh"

namespace hdc {

// Block size cap of the transform kernels (every stage loops over its
// butterflies, so any count works): 256 threads at up to 128 registers let
// two blocks share an SM.
constexpr int kMaxThreads = 256;
// Shared-memory budgets.  The fused residue kernel holds f, g and one
// ping-pong buffer of m elements (3 smem_len(m), 96 KiB at the largest m),
// which keeps two blocks per SM, so one block's loads and barriers overlap
// the other's arithmetic.  The strided-axis kernels hold a tile of ma x C
// elements and its ping-pong twin (2 smem_len(ma C)): C is chosen so a tile
// fits 64 KiB in FP32 (three blocks per SM) and 32 KiB in FP64
// (col_tile_target), and a single column may use up to 128 KiB.
constexpr int64_t kRowBytes = 112 * 1024;
constexpr int64_t kColTargetBytes = 64 * 1024;
constexpr int64_t kColMaxBytes = 128 * 1024;

// largest power-of-two-rounded m whose three buffers fit kRowBytes
template <typename T> constexpr int64_t max_row_fft() { return (int64_t)1 << (sizeof(cx<T>) == 16 ? 11 : 12); }
static_assert(3 * smem_len<cx<double>>(2048) * 16 <= kRowBytes, "FP64 row tile exceeds its budget");
static_assert(3 * smem_len<cx<float>>(4096) * 8 <= kRowBytes, "FP32 row tile exceeds its budget");
// Elements of a column tile: kColTargetBytes over its two buffers in FP32,
// half of that in FP64, whose column passes are bound by their arithmetic
// and run faster as more, smaller blocks (1024-element tiles of 128 threads:
// the 2^22 fold 5 % faster than with 2048).
template <typename T> constexpr int64_t col_tile_target()
{
    return (sizeof(T) == 8 ? kColTargetBytes / 2 : kColTargetBytes) / (2 * (int64_t)sizeof(cx<T>));
}
template <typename T> constexpr int64_t max_col_fft() { return kColMaxBytes / (2 * (int64_t)sizeof(cx<T>)); }

// Stages of an n-point transform: radix 8 first (16 first when r16), then 4,
// 2, 7, 5, 3, with the offsets of their twiddle sub-tables.
FftPlan make_fft_plan(int64_t n, bool r16 = false, bool r2 = false);
// The plan the kernels use for element type T.  FP32 transforms whose
// kernel is built with radix-16 stages (r16ok) take them where they save a
// stage: FP32 stages are bound by shared-memory passes, which radix 16 makes
// fewer.  FP64 transforms are bound by FP64 arithmetic, which the
// twiddle-merged radix-2/4/8 butterflies keep lowest, and never take them.
template <typename T> inline FftPlan fft_plan(int64_t n, bool r16ok = false)
{
    return make_fft_plan(n, sizeof(T) == 4 && r16ok);
}
// The plan of a transform whose latency matters more than its instruction
// count (a few blocks, each on one SM): in FP64, whose warp instructions
// issue at half a lane per clock per SM sub-partition, a radix-8 stage keeps
// a thread on one butterfly for about 72 FMAs while radix-2 stages, with the
// same FMAs per point in all (3 per point and stage in the twiddle-merged
// form), spread over four times the threads with 6 FMAs each; so FP64
// latency plans take radix 2 throughout the power-of-two part.  FP32 keeps
// its usual plan.
template <typename T> inline FftPlan fft_plan_latency(int64_t n)
{
    return make_fft_plan(n, false, sizeof(T) == 8);
}
// A row transform runs n / 8 threads (at most kMaxThreads): below 16
// kMaxThreads points a radix-16 stage would leave some of them idle, so rows
// take radix 16 from there on.  Column tiles hold a butterfly per column and
// take it at any size.
inline bool rows_r16(int64_t n) { return n >= 16 * (int64_t)kMaxThreads; }
// kernels with radix-16 stages exist for FP32 only
template <class V> constexpr bool kHas16 = sizeof(V) == 8;
template <class V> inline bool takes_r16(const FftPlan& fp) { return kHas16<V> && fp.nst > 0 && fp.rad[0] == 16; }

// ------------------------------------------------------- twiddle tables
// The convolution entry points only look their twiddle tables up: a missing
// table makes the call return HDC_ERR_NOT_PREPARED before anything is
// launched, so no convolution call allocates device memory or synchronises.
// The preparation calls (hdc_prepare*, plan creation, the tuners, batched
// plans) make the missing tables.  The mode belongs to the calling host
// thread; a TableScope sets it for its lifetime (scopes nest).
enum TableMode {
    kTablesLookup = 0,  // look up only (the default)
    kTablesCreate = 1,  // make missing tables, then launch as usual
    kTablesPrepare = 2  // make missing tables and launch nothing: the walk of
                        // a call by hdc_prepare*, whose launchers return right
                        // after fetching their tables (no pointer is read)
};
struct TableScope {
    int saved;
    explicit TableScope(int mode);
    ~TableScope();
};
int table_mode();
inline bool preparing() { return table_mode() == kTablesPrepare; }
// Set when a lookup finds no table (turned into HDC_ERR_NOT_PREPARED by the
// entry point, which clears it).
bool& tables_missing();
// 256 MiB a tuner writes before each timed replay to evict L2 (made on first
// use in a table-making mode, like a table); *bytes gets its size.
void* tuning_flush_buffer(size_t* bytes);

// ------------------------------------------------------ launch statistics
// Every launcher counts its launches and the model flops / algorithmic
// bytes of the launch; when timing is on it also brackets the launch with
// CUDA events on its stream.

// K_FOLD_TMA counts the launches of k_fold_fft_cols that stage their tiles
// with TMA copies (K_FOLD_FFT_COLS those on plain loads).
enum KernelId { K_TWIDDLE = 0, K_RESIDUE_ROWS, K_FOLD_FFT_COLS, K_IFFT_COLS, K_UNFOLD, K_BATCHED, K_IFFT_UNFOLD,
                K_FOLD_TMA, K_CLUSTER, K_HERMITIAN_ROWS, K_COUNT };

struct LaunchScope {
    int kid;
    cudaStream_t st;
    cudaEvent_t e0;
    LaunchScope(int kid, cudaStream_t st, double flops, double bytes);
    ~LaunchScope();
};

// 5 n log2(n): the flop count convention of one n-point complex FFT.
double fft_flops(double n);

// Twiddle table zeta_n^k, k < n, of dtype T on the current device (cached).
template <typename T> const cx<T>* twiddles(int64_t n, cudaError_t* err);
// The packed per-stage tables of the n-point transform's plan (FftPlan::toff),
// plain (lf = false) or in the scale-tangent form of the twiddle-merged
// butterflies (lf = true, see lf_bfly): what fft_smem reads; of the plan
// fft_plan<T>(n, r16ok).
template <typename T> const cx<T>* twiddles_fft(int64_t n, bool lf, cudaError_t* err, bool r16ok = false);
// The same tables for any plan of the transform (cached per plan shape).
template <typename T> const cx<T>* twiddles_fft_plan(const FftPlan& fp, bool lf, cudaError_t* err);
// zeta_N^k for the folds and unfolds: one table, or two for a large N (TwTab).
template <typename T> TwTab<cx<T>> tw_table(int64_t N, cudaError_t* err);
// zeta_{ma Cn}^{l c} at c ma + l (l < ma, c < Cn): the four-step twiddles of an
// ma x Cn split in the order a column tile reads them.
template <typename T> const cx<T>* twiddles_colmajor(int64_t ma, int64_t Cn, cudaError_t* err);

// ------------------------------------------------------------ launchers

// Fused residue kernel over rows: for every row b < B and residue
// r = r0 + rr (rr < D, r < q): fold the row of f and g (period m, p blocks,
// valid elements j < Lf of f at stride ld_f, j < L of g at stride ld_g),
// m-point FFTs, product, inverse FFT, and write the unscaled result to
// h + ((rr * B + b) * m).
template <typename T>
cudaError_t launch_residue_rows(const cx<T>* f, const cx<T>* g, cx<T>* h, int64_t B, int64_t ld_f, int64_t ld_g,
                                int64_t Lf, int64_t L, int64_t m, int64_t p, int64_t q, int64_t r0, int64_t D,
                                cudaStream_t st);

// Fused residue kernel with residue matching (unequal lengths): g rows at
// mg = lam mf points (pg blocks, qg residues, Lg valid), f rows at mf points
// (pf blocks, lam qg residues, Lf valid); residues rg = r0 + rr of g, each
// with its lam matching residues of f; unscaled mg-point results to
// h + ((rr * B + b) * mg).
template <typename T>
cudaError_t launch_residue_rows_lam(const cx<T>* f, const cx<T>* g, cx<T>* h, int64_t B, int64_t ld_f,
                                    int64_t ld_g, int64_t Lf, int64_t Lg, int64_t mf, int64_t lam, int64_t pf,
                                    int64_t pg, int64_t qg, int64_t r0, int64_t D, cudaStream_t st);

// Multi-convolution rows: like launch_residue_rows for nin (<= kMaxInputs)
// equal-length inputs xs[i] (row stride ld, L valid): per residue the
// product of all nin transforms (op 0) or the sum of the pairwise products
// F_0 F_1 + F_2 F_3 + ... (op 1), unscaled results to h + ((rr * B + b) * m).
template <typename T>
cudaError_t launch_residue_rows_multi(const cx<T>* const* xs, int nin, int op, cx<T>* h, int64_t B, int64_t ld,
                                      int64_t L, int64_t m, int64_t p, int64_t q, int64_t r0, int64_t D,
                                      cudaStream_t st);

// One input of the strided fold + column FFT pass.  Array view
// x[b][a][c] (batch stride bstride) with a < A (axis), c < Cn; element valid
// iff a * Cn + c < Lvalid; p fold blocks, q residues.  Residue block (l, rr),
// l < lam, rr < D, is residue r0 + rr + l * rmul; its output row i goes to
// row i * lam + l of y[rr][b] (rows of Cn, lam * ma rows per (rr, b)).  The
// equal-length case is lam = 1, rmul = 0.
template <typename T> struct ColSide {
    const cx<T>* x;
    cx<T>* y;
    int64_t bstride, Lvalid;
    int p, q, rmul, lam;
    int rneg = 0; // 1: residue block rr is residue (q - (r0 + rr)) mod q
};

// Fold along a strided axis + FFT of size ma over that axis, for nside <=
// kMaxInputs inputs (one launch; with more than one, all have lam = 1),
// column tile of width C.
// Fold twiddle zeta_Nf^{r (i cs + c cc)}; if post != 0 the transformed
// value is multiplied by zeta_{Nf/q}^{l c} (the inner twiddle of a split
// ma * Cn transform).
template <typename T>
cudaError_t launch_fold_fft_cols(const ColSide<T>* sides, int nside, int64_t B, int64_t Cn, int64_t ma, int64_t Nf,
                                 int64_t cs, int64_t cc, int64_t r0, int64_t D, int post, cudaStream_t st);

// Real inputs (packed z = f + i g; only the residues r <= q / 2 are kept,
// each with its conjugate partner r' = (q - r) mod q):
//  launch_pack_real      z[i] = f[i] + i g[i], n elements;
//  launch_residue_rows_real  fused rows: kept residues r0 .. r0 + Dg - 1 of
//                        every row of z (stride ld, L valid), unscaled H
//                        transforms' inverses to h[rr][b][0..m);
//  launch_rows_real_pair split rows: row l1 of ya[rr][b] with the mirrored
//                        row of yb[rr][b] (the partners' column pass; ya for
//                        a self-paired residue, whose partner pass is
//                        skipped), into yh (distinct from ya and yb);
//  launch_pair_rows_real outer axis of N-D: wf <- F, wg <- G elementwise from
//                        wa and the mirrored rows of wb (of wa when
//                        self-paired);
//  launch_unfold_real    the weighted real part of the kept residues'
//                        contributions, real output.
template <typename T> cudaError_t launch_pack_real(const T* f, const T* g, cx<T>* z, int64_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_residue_rows_real(const cx<T>* z, cx<T>* h, int64_t B, int64_t ld, int64_t L, int64_t m,
                                     int64_t p, int64_t q, int64_t r0, int64_t Dg, cudaStream_t st);
template <typename T>
cudaError_t launch_rows_real_pair(const cx<T>* ya, const cx<T>* yb, cx<T>* yh, int64_t B, int64_t m1, int64_t m2,
                                  int64_t q, int64_t r0, int64_t Dg, cudaStream_t st);
template <typename T>
cudaError_t launch_pair_rows_real(const cx<T>* wa, const cx<T>* wb, cx<T>* wf, cx<T>* wg, int64_t B, int64_t Cn,
                                  int64_t m0, int64_t q, int64_t r0, int64_t Dg, cudaStream_t st);
template <typename T>
cudaError_t launch_unfold_real(T* out, const cx<T>* h, int64_t B, int64_t bstride, int64_t Cn, int64_t ma,
                               int64_t p, int64_t q, int64_t Nf, int64_t cs, int64_t cc, int64_t lo, int64_t hi,
                               int64_t r0, int64_t Dg, int first, int last, double scale, cudaStream_t st);

// Whole 1-D convolutions of B short rows on thread-block clusters (one
// cluster per row): residues [r_lo, r_hi) of f and g (row strides ld_f,
// ld_g, L valid elements, m-point transforms, p fold blocks, q residues)
// from fold to unfold in one launch, the outputs [lo, hi) of each row
// written once (times scale) to out (row stride ldo).  cluster_shape tells
// whether an m-point residue (pout = ceil(hi / m) output blocks, q residues,
// p fold blocks) fits a cluster: C blocks, m = m1 m2 with C dividing both;
// *stage (optional): the inputs fit in shared memory too; *warp (optional):
// the transforms run as warp shuffles (m1, m2 powers of two up to 64).
template <typename T>
bool cluster_shape(int64_t m, int64_t pout, int64_t q, int64_t p, int* C, int64_t* m1, int64_t* m2,
                   bool* stage = nullptr, bool* warp = nullptr);
int cluster_route_mode();
template <typename T>
cudaError_t launch_conv_cluster(const cx<T>* f, const cx<T>* g, cx<T>* out, int64_t B, int64_t ld_f, int64_t ld_g,
                                int64_t ldo, int64_t L, int64_t lo, int64_t hi, int64_t m, int64_t p, int64_t q,
                                int64_t r_lo, int64_t r_hi, double scale, cudaStream_t st);

// Inner axis of the centered Hermitian 2-D convolution (K = c + 1 stored
// ky >= 0 values per row): rows (rr, b, l) of wf / wg at ((rr B + b) mx + l) K
// hold F_s, G_s of outer bin x = qx l + r0 + rr (Nx = qx mx points); per pair
// of rows the packed fold and my-point transforms of every ky residue (qy
// residues, ky laid out cyclically over Ny = qy my >= 3c + 1 points), the
// real products, one packed inverse transform and unfold of the outputs
// ky in [-c, c], split by symmetry; the
// k >= 0 halves times zeta_Nx^{2 c x} and 1 / (qy my) go to the same rows of
// wh.  nblk = (outer residues of the pass) x B.
template <typename T>
cudaError_t launch_hermitian_rows(const cx<T>* wf, const cx<T>* wg, cx<T>* wh, int64_t nblk, int64_t B, int64_t mx,
                                  int64_t K, int64_t my, int64_t qy, int64_t Nx, int64_t qx, int64_t r0,
                                  cudaStream_t st);

// In-place inverse FFT of size ma along the strided axis of y[rr][b][l][c],
// preceded by multiplication with conj(zeta_{Nf/q}^{l c}) if pre != 0.
template <typename T>
cudaError_t launch_ifft_cols(cx<T>* y, int64_t B, int64_t Cn, int64_t ma, int64_t q, int64_t Nf,
                             int64_t D, int pre, cudaStream_t st);

// Inverse column FFTs and unfold in one pass for one residue per pass when
// the column tiles of all rows give at least two blocks per SM: each block
// takes a column tile of one row through its inverse FFT and adds its unfold
// contribution to the outputs only it covers, so the residue's result never
// goes back to memory (the kernel also runs several residues in order, but
// that was measured slower than the two passes); otherwise launch_ifft_cols
// then launch_unfold.  Arguments as for those two.
template <typename T>
cudaError_t launch_ifft_unfold(cx<T>* y, cx<T>* out, int64_t B, int64_t bstride, int64_t Cn, int64_t ma, int64_t p,
                               int64_t q, int64_t Nf, int64_t cs, int64_t cc, int64_t lo, int64_t hi, int64_t r0,
                               int64_t D, int first, int last, double scale, int pre, cudaStream_t st);

// Unfold-accumulate: the output at lin = (t ma + i) Cn + c, t < p, kept iff
// lo <= lin < hi and stored at out[b * bstride + lin - lo], gets
// sum_{rr} conj(zeta_Nf^{r (i cs + c cc)}) conj(zeta_q^{r t}) h[rr][b][i][c];
// added to the previous contents unless first, scaled by `scale` if last.
template <typename T>
cudaError_t launch_unfold(cx<T>* out, const cx<T>* h, int64_t B, int64_t bstride, int64_t Cn,
                          int64_t ma, int64_t p, int64_t q, int64_t Nf, int64_t cs, int64_t cc,
                          int64_t lo, int64_t hi, int64_t r0, int64_t D, int first, int last, double scale,
                          cudaStream_t st);

// The same launches with caller-provided twiddle tables (no library cache):
// twN = zeta_{q m}^k (q m entries), twm / twml the packed stage tables of the
// m-point transform (launch_twiddle_fft_into), twNf as in launch_unfold;
// launch_twiddle_into fills a table of n entries on `st`.
template <typename T> cudaError_t launch_twiddle_into(cx<T>* tw, int64_t n, cudaStream_t st);
// Fills a packed table of fp.tlen entries (see FftPlan) on `st`.
template <typename T> cudaError_t launch_twiddle_fft_into(cx<T>* tw, const FftPlan& fp, bool lf, cudaStream_t st);
template <typename T>
cudaError_t launch_residue_rows_tw(const cx<T>* f, const cx<T>* g, cx<T>* h, int64_t B, int64_t ld_in,
                                   int64_t L, int64_t m, int64_t p, int64_t q, int64_t r0, int64_t D,
                                   const cx<T>* twN, const cx<T>* twm, const cx<T>* twml, cudaStream_t st);
template <typename T>
cudaError_t launch_unfold_tw(cx<T>* out, const cx<T>* h, int64_t B, int64_t bstride, int64_t Cn, int64_t ma,
                             int64_t p, int64_t q, int64_t Nf, int64_t cs, int64_t cc, int64_t Lvalid,
                             int64_t r0, int64_t D, int first, int last, double scale, const cx<T>* twNf,
                             cudaStream_t st);

} // namespace hdc

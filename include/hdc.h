/*
 * hdc.h -- hybrid dealiased convolution on GB300 (sm_103a): the C ABI.
 *
 * The library computes the first L outputs of the linear convolution of two
 * length-L complex inputs per axis (Section 2.3, Eq. 4, read with inputs of
 * length L, zero beyond):
 *
 *     h_k = sum_{j=0}^{k} f_j g_{k-j},            k = 0 .. L-1,
 *
 * in 1, 2 or 3 dimensions, by the residue decomposition of Section 2.2:
 * with zeta_n = exp(2 pi i / n), N = q m, j = t m + s, k = q l + r,
 *
 *   forward (Eq. 1):  F_{q l + r} = sum_s zeta_m^{l s} zeta_N^{r s} sum_t zeta_q^{r t} f_{t m + s}
 *   backward (Eq. 2): f_{t m + s} = (1/N) sum_r zeta_q^{-t r} zeta_N^{-s r} sum_l zeta_m^{-s l} F_{q l + r}
 *
 * i.e. for every residue r: a twiddled fold of the p input blocks, an m-point
 * FFT, the pointwise product of the two transforms (the convolution theorem,
 * Section 2.4), an m-point inverse FFT and a twiddled unfold that
 * accumulates the first L outputs.  Explicit padding (m >= M, p = q = 1,
 * Section 3.1), implicit padding (L = p m, M = q m, Section 3.2) and hybrid
 * padding (Section 3.3) are parameter choices of the same call.
 *
 * Parameters per axis (Section 2.5): L (input length), M (padded length,
 * M >= 2L-1 for an alias-free result), m (FFT size), p = ceil(L/m) and
 * q = ceil(M/m) (pass 0 to derive them; larger values are accepted), D
 * (residues computed per pass, 1..q; 0 means q), I (in place: h may alias f).
 *
 * Conventions for every entry point:
 *  - Arrays are interleaved complex (re, im), row-major, last axis fastest:
 *    HDC_C128 = complex<double> (16 B), HDC_C64 = complex<float> (8 B); the
 *    memory layout of torch.complex128 / torch.complex64.  A batch of B
 *    problems is B consecutive arrays.
 *  - f, g, h and the workspace are DEVICE pointers owned by the caller,
 *    16-byte aligned, on the current CUDA device.  f and g are read-only
 *    unless inplace = 1, in which case h may equal f or g.
 *  - The convolution calls allocate nothing and never synchronise.  The
 *    twiddle tables they read (zeta_n^k for exact integer k, one FP64
 *    sincospi each, made once per (n, dtype, device) and kept until
 *    hdc_release_caches()) are made by the preparation calls: hdc_prepare*
 *    (one per kind of convolution call, same arguments minus the data),
 *    hdc_plan_create, the tuners and hdc_batched_create.  A convolution call
 *    whose tables are missing returns HDC_ERR_NOT_PREPARED and launches
 *    nothing.  The caller allocates the workspace; query its size with
 *    hdc_workspace_size().
 *  - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default)
 *    and is asynchronous; nothing is synchronised.
 *  - Every error is a return code (hdc_status).  Nothing throws across the
 *    ABI, nothing traps on the device.  Invalid parameters are rejected on
 *    the host before any launch.
 */
#ifndef HDC_H
#define HDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HDC_MAX_DIMS 3

typedef enum hdc_status {
    HDC_OK = 0,
    HDC_ERR_PARAM = -1,            /* inconsistent (L, M, m, p, q, D) or bad pointer/size  */
    HDC_ERR_ALIAS = -2,            /* M < 2L-1: the result would contain aliases (Section 3.1) */
    HDC_ERR_UNSUPPORTED_SIZE = -3, /* m not of the form 2^a 3^b 5^c 7^d, or beyond the limits */
    HDC_ERR_DTYPE = -4,            /* unknown hdc_dtype                                     */
    HDC_ERR_ALLOC = -5,            /* twiddle-table allocation failed                       */
    HDC_ERR_CUDA = -6,             /* a CUDA runtime call or kernel launch failed           */
    HDC_ERR_TIMEOUT = -7,          /* a bounded device-side wait gave up                    */
    HDC_ERR_NOT_TUNED = -8,        /* no tuning record / predictor for the request          */
    HDC_ERR_WORKSPACE = -9,        /* workspace missing or smaller than required            */
    HDC_ERR_NOT_PREPARED = -10     /* twiddle tables not made: call hdc_prepare* first      */
} hdc_status;

typedef enum hdc_dtype {
    HDC_C64 = 0,   /* complex<float>  */
    HDC_C128 = 1   /* complex<double> */
} hdc_dtype;

/* How a plan chooses (m, p, q, D) per axis. */
typedef enum hdc_mode {
    HDC_FIXED = 0,            /* the caller's m (and D) per axis                    */
    HDC_TUNE_EXHAUSTIVE = 1,  /* grid search on the device (Section 4.2), cached     */
    HDC_PREDICT_MLP = 2,      /* learned predictor of the parameters                 */
    HDC_EXPLICIT = 3,         /* explicit padding m = nextgood(M), p = q = 1 (3.1)   */
    HDC_TUNE_CACHED_ONLY = 4, /* tuning database only; HDC_ERR_NOT_TUNED if absent   */
    HDC_PREDICT_MLP_SEARCH = 5, /* time the predictor's 3 best classes per axis and  */
                                /* the q-neighbours of its best two                   */
    HDC_TUNE_RANDOM = 6,        /* random search (Section 4.3, A1): a quarter of the  */
                                /* candidates, cached                                 */
    HDC_TUNE_PROXY = 7          /* per axis, search the rectangle with the other axes */
                                /* cut to 32 points (Section 6.3 heuristic), cached   */
} hdc_mode;

/* One parameter choice of one axis and its measured time. */
typedef struct hdc_tuple {
    int64_t m, p, q, D;
    double model_flops;  /* F1 = q (15 m log2 m + 6 m + 24 L) + 2 L of the axis   */
    double ms;           /* median device time of the whole convolution, or -1    */
} hdc_tuple;

/* Opaque, library-owned plan (host memory only). */
typedef struct hdc_plan hdc_plan;

/* ------------------------------------------------------------ host helpers
 * No GPU needed. */

/* Human-readable text for an hdc_status. Never NULL. */
const char* hdc_strerror(int status);

/* The cudaError_t code (0 if none yet) behind the most recent HDC_ERR_CUDA
 * that a convolution entry point returned, and its name (cudaGetErrorName). */
int hdc_last_cuda_error(void);
const char* hdc_last_cuda_error_name(void);

/* Library version as major*10000 + minor*100 + patch. */
int hdc_version(void);

/* 1 if n >= 1 has no prime factor above 7 (an FFT size this library runs,
 * the 2^a 3^b 5^c 7^d sizes of Section 3.1 and Section 5.1), else 0. */
int hdc_is_good_size(int64_t n);

/* Smallest 2^a 3^b 5^c 7^d >= n (n >= 1); -1 on overflow or n < 1. */
int64_t hdc_next_good_size(int64_t n);

/* Section 2.5: p = ceil(L/m), q = ceil(M/m), the smallest integers with
 * p m >= L and q m >= M.  Returns HDC_ERR_PARAM for L, M, m < 1. */
int hdc_derive_params(int64_t L, int64_t M, int64_t m, int64_t* p, int64_t* q);

/* Explicit padding (Section 3.1): m = smallest good size >= M, p = q = 1. */
int hdc_explicit_params(int64_t L, int64_t M, int64_t* m, int64_t* p, int64_t* q);

/* Check one axis.  p, q, D may be 0 (derived: p = ceil(L/m), q = ceil(M/m),
 * D = q); the resolved values are written back through p_out, q_out, D_out
 * when those are non-NULL.  Errors: HDC_ERR_PARAM (L, M, m < 1, p m < L,
 * q m < M, D > q), HDC_ERR_ALIAS (M < 2L-1), HDC_ERR_UNSUPPORTED_SIZE (m not
 * 7-smooth, m or q m beyond hdc_max_fft_size / hdc_max_padded_size),
 * HDC_ERR_DTYPE. */
int hdc_validate_axis(int64_t L, int64_t M, int64_t m, int64_t p, int64_t q,
                      int64_t D, int dtype, int64_t* p_out, int64_t* q_out,
                      int64_t* D_out);

/* Largest FFT size m and padded size q m accepted for a dtype: m up to
 * 2^23 for complex<double> and 2^25 for complex<float> (the product of the
 * row and column tile limits; a larger m, or one that does not factor as a
 * row length <= 2048 / 4096 times a column length <= 4096 / 8192, is
 * HDC_ERR_UNSUPPORTED_SIZE), q m up to 2^25 / 2^26.  An axis that has inner
 * axes (all but the last of a 2-D / 3-D call) runs its m-point FFT in one
 * column tile: m <= hdc_max_outer_fft_size (4096 for complex<double>, 8192
 * for complex<float>), else HDC_ERR_UNSUPPORTED_SIZE. */
int64_t hdc_max_fft_size(int dtype);
int64_t hdc_max_padded_size(int dtype);
int64_t hdc_max_outer_fft_size(int dtype);

/* Kinds of shared-memory transform, for hdc_fft_stages. */
enum hdc_fft_kind {
    HDC_FFT_ROWS = 0,   /* residue rows: 1-D rows, the split's rows, the last axis */
    HDC_FFT_COLS = 1,   /* column tiles: the split's columns, the outer axes       */
    HDC_FFT_OTHER = 2   /* rows of the real-input, unequal-length and multi-
                           convolution kernels; rows and columns of the batched
                           kernel                                                 */
};

/* The stages of the n-point FFT (Section 2.2's radix-2 split generalised to
 * mixed radix, Stockham order) that a kernel of the given kind runs:
 * writes the radices, first stage first, to radices[0..cap) and returns
 * their number (0 for n = 1); their product is n.  Radix 8 first, then 4,
 * 2, 7, 5, 3; complex<float> transforms of kind HDC_FFT_COLS, and of kind
 * HDC_FFT_ROWS from 4096 points on, start with radix-16 stages where those
 * save a stage on the power-of-two part 2^e of n (ceil(e/4) < ceil(e/3)).
 * Host only, no GPU needed.  Errors: HDC_ERR_PARAM (radices NULL, cap < 0,
 * cap below the stage count, kind unknown), HDC_ERR_UNSUPPORTED_SIZE (n < 1,
 * n not 7-smooth, n above the kind's tile: 2048 / 4096 points for rows,
 * hdc_max_outer_fft_size for columns), HDC_ERR_DTYPE. */
int hdc_fft_stages(int64_t n, int dtype, int kind, int* radices, int cap);

/* Bytes of device workspace an N-D call needs (dims in 1..3; arrays of
 * length dims; p/q/D entries may be 0 = derive).  Writes *bytes. */
int hdc_workspace_size(int dims, const int64_t* L, const int64_t* M,
                       const int64_t* m, const int64_t* p, const int64_t* q,
                       const int64_t* D, int dtype, int64_t batch, int inplace,
                       size_t* bytes);

/* ---------------------------------------------------------- convolutions */

/* 1-D (Section 2.2-3.3): `batch` independent convolutions of length L.
 * f, g, h: batch x L complex.  Workspace of hdc_workspace_size(1, ...). */
int hdc_conv1d(const void* f, const void* g, void* h, int64_t L, int64_t M,
               int64_t m, int64_t p, int64_t q, int64_t D, int inplace,
               int dtype, int64_t batch, void* workspace, size_t ws_bytes,
               void* stream);

/* 2-D (Section 3.6, recursion over axes): f, g, h: batch x L[0] x L[1].
 * Axis 0 is transformed by residues first; the inner 1-D convolution along
 * axis 1 runs on each of its m[0] transformed rows per residue. */
int hdc_conv2d(const void* f, const void* g, void* h, const int64_t L[2],
               const int64_t M[2], const int64_t m[2], const int64_t p[2],
               const int64_t q[2], const int64_t D[2], int inplace, int dtype,
               int64_t batch, void* workspace, size_t ws_bytes, void* stream);

/* 3-D (Section 3.6): f, g, h: batch x L[0] x L[1] x L[2]. */
int hdc_conv3d(const void* f, const void* g, void* h, const int64_t L[3],
               const int64_t M[3], const int64_t m[3], const int64_t p[3],
               const int64_t q[3], const int64_t D[3], int inplace, int dtype,
               int64_t batch, void* workspace, size_t ws_bytes, void* stream);

/* Any of the above by rank (dims in 1..3). */
int hdc_convnd(int dims, const void* f, const void* g, void* h,
               const int64_t* L, const int64_t* M, const int64_t* m,
               const int64_t* p, const int64_t* q, const int64_t* D,
               int inplace, int dtype, int64_t batch, void* workspace,
               size_t ws_bytes, void* stream);

/* The same convolution on HOST buffers f, g, h (pinned for asynchronous
 * copies; pageable works but serialises): copies f and g into the device
 * workspace, convolves there and copies the result back into h, all on
 * `stream`; synchronise the stream before reading h.  The device workspace
 * holds both device copies, the result and the convolution workspace: size
 * it with hdc_workspace_size_host().  inplace is not accepted here. */
int hdc_workspace_size_host(int dims, const int64_t* L, const int64_t* M,
                            const int64_t* m, const int64_t* p, const int64_t* q,
                            const int64_t* D, int dtype, int64_t batch,
                            size_t* bytes);
int hdc_convnd_host(int dims, const void* f_host, const void* g_host,
                    void* h_host, const int64_t* L, const int64_t* M,
                    const int64_t* m, const int64_t* p, const int64_t* q,
                    const int64_t* D, int dtype, int64_t batch,
                    void* dev_workspace, size_t ws_bytes, void* stream);

/* Output windows (Section 3.1 read for any slice of the linear
 * convolution): per axis, the outputs [o, o + Lw) of the full linear
 * convolution (length 2L - 1) instead of the first L.  The window is
 * alias-free when M >= 2L - 1 - o and o + Lw <= q m (else HDC_ERR_ALIAS);
 * o = 0, Lw = 2L - 1 with M >= 2L - 1 gives the whole linear convolution.
 * h: batch x prod(Lw) complex.  Same conventions as hdc_convnd (no
 * in-place mode). */
int hdc_workspace_size_window(int dims, const int64_t* L, const int64_t* M,
                              const int64_t* m, const int64_t* p,
                              const int64_t* q, const int64_t* D,
                              const int64_t* o, const int64_t* Lw, int dtype,
                              int64_t batch, size_t* bytes);
int hdc_convnd_window(int dims, const void* f, const void* g, void* h,
                      const int64_t* L, const int64_t* M, const int64_t* m,
                      const int64_t* p, const int64_t* q, const int64_t* D,
                      const int64_t* o, const int64_t* Lw, int dtype,
                      int64_t batch, void* workspace, size_t ws_bytes,
                      void* stream);

/* Unequal lengths with residue matching (Section 3.5, the final algorithms
 * for one and for N dimensions).  Per axis i, f has Lf[i] elements and g
 * Lg[i]; f is transformed at m[i] points and g at lam[i] m[i] points
 * (lam[i] >= 1; lam = 1 shares one transform size).  Derived per axis:
 * pf = ceil(Lf / m), pg = ceil(Lg / (lam m)), qg = ceil(M / (lam m)),
 * qf = lam qg, N = qg lam m = qf m.  Residue rg of g pairs DFT bin
 * lam lf + l of its lam m-point transform with bin lf of residue qg l + rg of
 * f (l < lam), since qg (lam lf + l) + rg = qf lf + (qg l + rg).  D[i] is the
 * number of g residues per pass (1..qg; 0 or NULL: all).
 *
 * Output: per axis the window [o, o + Lw) of the linear convolution (length
 * Lf + Lg - 1); o = NULL means 0, Lw = NULL means Lg (Eq. 4's first outputs
 * for the longer input).  Alias-free when M >= Lf + Lg - 1 - o and
 * o + Lw <= N (else HDC_ERR_ALIAS); M = NULL (or M[i] <= 0) takes the least
 * such M.  Either input may be the longer one, but the shorter one should be
 * f so it gets the smaller transform.
 *
 * m and lam m must be 2^a 3^b 5^c 7^d; lam m within hdc_max_fft_size, and for
 * every axis but the last within hdc_max_outer_fft_size; a split transform
 * (lam m above 2048 points for complex<double>, 4096 for complex<float>)
 * needs a factor m1 of lam m divisible by lam with lam m / m1 within the
 * row limit (else HDC_ERR_UNSUPPORTED_SIZE).
 *
 * f: batch x prod(Lf), g: batch x prod(Lg), h: batch x prod(Lw), complex,
 * row-major, device memory, distinct buffers (h may alias neither input:
 * HDC_ERR_PARAM).  The workspace (device, caller-owned, at least the size
 * hdc_workspace_size_unequal reports) is only used during the call.  Runs
 * asynchronously on `stream`. */
int hdc_validate_unequal_axis(int64_t Lf, int64_t Lg, int64_t M, int64_t m,
                              int64_t lam, int64_t D, int dtype, int64_t* pf,
                              int64_t* pg, int64_t* qg, int64_t* D_out);
int hdc_workspace_size_unequal(int dims, const int64_t* Lf,
                               const int64_t* Lg, const int64_t* M,
                               const int64_t* m, const int64_t* lam,
                               const int64_t* D, const int64_t* o,
                               const int64_t* Lw, int dtype, int64_t batch,
                               size_t* bytes);
int hdc_convnd_unequal(int dims, const void* f, const void* g, void* h,
                       const int64_t* Lf, const int64_t* Lg, const int64_t* M,
                       const int64_t* m, const int64_t* lam, const int64_t* D,
                       const int64_t* o, const int64_t* Lw, int dtype,
                       int64_t batch, void* workspace, size_t ws_bytes,
                       void* stream);

/* Multi-convolution of n arrays (n = 2..8; the paper extends the method
 * to N arrays), all inputs of one shape, first L outputs per axis, with one
 * of two operators applied per DFT index of each residue:
 *   HDC_MULTI_PRODUCT: the n-fold convolution x_0 * x_1 * ... * x_{n-1}
 *     (product of all n transforms); its result has length n (L - 1) + 1
 *     per axis, so M >= n (L - 1) + 1 (else HDC_ERR_ALIAS);
 *   HDC_MULTI_DOT: the sum of pairwise convolutions
 *     x_0 * x_1 + x_2 * x_3 + ... (n even, else HDC_ERR_PARAM), M >= 2L - 1.
 * Per residue every input is folded and transformed (Eq. 1), the operator
 * is applied, and one inverse transform and unfold follow (Eq. 2).  M =
 * NULL (or M[i] <= 0) takes the least alias-free M.  m, p, q, D as in
 * hdc_convnd.  inputs: n device pointers, each batch x prod(L) complex; h:
 * batch x prod(L), distinct from every input (else HDC_ERR_PARAM).
 * Workspace: hdc_workspace_size_multi. */
enum hdc_multi_op { HDC_MULTI_PRODUCT = 0, HDC_MULTI_DOT = 1 };
int hdc_workspace_size_multi(int dims, int n, int op, const int64_t* L,
                             const int64_t* M, const int64_t* m,
                             const int64_t* p, const int64_t* q,
                             const int64_t* D, int dtype, int64_t batch,
                             size_t* bytes);
int hdc_convnd_multi(int dims, int n, int op, const void* const* inputs, void* h,
                     const int64_t* L, const int64_t* M, const int64_t* m,
                     const int64_t* p, const int64_t* q, const int64_t* D,
                     int dtype, int64_t batch, void* workspace,
                     size_t ws_bytes, void* stream);

/* Convolution of real inputs (the paper's future work on the real case,
 * Section 7): f, g and h are REAL arrays (dtype HDC_C128: double, HDC_C64:
 * float), batch x prod(L), first L outputs per axis, same (L, M, m, p, q)
 * rules as hdc_convnd.  The two inputs are packed as one complex sequence
 * z = f + i g; since f and g are real, F and G at DFT index K follow from Z
 * at K and at -K, and -K of residue r (axis 0) lies in residue
 * (q - r) mod q.  Only the residues r <= q / 2 of axis 0 are formed, each
 * from its pair of transforms, and each output is the real part of their
 * contributions with the partner's folded in (factor 2 unless r = 0 or
 * 2 r = q): two forward and one inverse transform per pair of residues
 * instead of six.  Inner axes (N-D) run the complex convolution of the F
 * and G rows.  D[0] counts kept residues per pass (clamped to q / 2 + 1).
 * Workspace (device, caller-owned): hdc_workspace_size_real; h distinct
 * from f and g (else HDC_ERR_PARAM). */
int hdc_workspace_size_real(int dims, const int64_t* L, const int64_t* M,
                            const int64_t* m, const int64_t* p,
                            const int64_t* q, const int64_t* D, int dtype,
                            int64_t batch, size_t* bytes);
int hdc_convnd_real(int dims, const void* f, const void* g, void* h,
                    const int64_t* L, const int64_t* M, const int64_t* m,
                    const int64_t* p, const int64_t* q, const int64_t* D,
                    int dtype, int64_t batch, void* workspace,
                    size_t ws_bytes, void* stream);

/* The share of residues [r_lo, r_hi) of axis 0 (0 <= r_lo < r_hi <= q[0]):
 * the outer sum of Eq. 2 restricted to that range, scaled by 1/N, so the
 * shares of disjoint ranges add up to the convolution.  Residues are
 * independent until that sum (Section 2.2), which is how a convolution is
 * split over several GPUs: each computes one range, then one sum-reduction
 * of the outputs.  Same arguments as hdc_convnd (no in-place mode; the
 * workspace of hdc_workspace_size is enough). */
int hdc_convnd_residues(int dims, const void* f, const void* g, void* h,
                        const int64_t* L, const int64_t* M, const int64_t* m,
                        const int64_t* p, const int64_t* q, const int64_t* D,
                        int64_t r_lo, int64_t r_hi, int dtype, int64_t batch,
                        void* workspace, size_t ws_bytes, void* stream);

/* Centered Hermitian 2-D convolution (the paper names the Hermitian case as
 * prior work, Section 1, and future work, Section 7; this is the reading
 * used here): f and g are the non-redundant halves of two Hermitian-
 * symmetric spectra on |kx|, |ky| <= K-1 -- arrays (2K-1) x K, row
 * kx + K - 1, column ky >= 0, the other half being f(-k) = conj(f(k)) --
 * and h (same layout) gets h_k = sum_{p, k-p in the box} f_p g_{k-p} for
 * |kx| <= K-1, 0 <= ky <= K-1: the dealiased product of two real fields.
 * Computed as the linear convolution of the index-shifted full spectra
 * with padding M = 3K - 2 per axis (the 3/2 ratio; m per axis, e.g. m = K
 * gives q = 3), keeping the windows [K-1, 3K-3] and [2K-2, 3K-3].
 * h may alias neither input. */
int hdc_workspace_size_hermitian(int64_t K, const int64_t* m, const int64_t* D,
                                 int dtype, int64_t batch, size_t* bytes);
int hdc_conv2d_hermitian(const void* f, const void* g, void* h, int64_t K,
                         const int64_t* m, const int64_t* D, int dtype,
                         int64_t batch, void* workspace, size_t ws_bytes,
                         void* stream);

/* ---------------------------------------------------------- preparation
 * Make, on the current device, every twiddle table the matching convolution
 * call with these arguments reads (the zeta_N^k of the folds and unfolds,
 * N = q m per axis, and the per-stage tables of the m-point transforms of
 * its route; Section 2.2).  This is where the library allocates: each
 * missing table is a cudaMalloc and a kernel on a private stream that is
 * waited for, so prepare before any stream capture.  Tables already made
 * cost a lookup.  Nothing is launched on the caller's streams and no data
 * pointer is needed.  The batch count matters (it selects the route).
 *   hdc_prepare           for hdc_convnd / conv1d / conv2d / conv3d,
 *                         hdc_convnd_host and hdc_convnd_residues
 *   hdc_prepare_window    for hdc_convnd_window
 *   hdc_prepare_hermitian for hdc_conv2d_hermitian
 *   hdc_prepare_unequal   for hdc_convnd_unequal
 *   hdc_prepare_multi     for hdc_convnd_multi
 *   hdc_prepare_real      for hdc_convnd_real
 * Errors: those of the convolution call's parameter checks, HDC_ERR_CUDA. */
int hdc_prepare(int dims, const int64_t* L, const int64_t* M, const int64_t* m,
                const int64_t* p, const int64_t* q, const int64_t* D, int dtype,
                int64_t batch);
int hdc_prepare_window(int dims, const int64_t* L, const int64_t* M,
                       const int64_t* m, const int64_t* p, const int64_t* q,
                       const int64_t* D, const int64_t* o, const int64_t* Lw,
                       int dtype, int64_t batch);
int hdc_prepare_hermitian(int64_t K, const int64_t* m, const int64_t* D,
                          int dtype, int64_t batch);
int hdc_prepare_unequal(int dims, const int64_t* Lf, const int64_t* Lg,
                        const int64_t* M, const int64_t* m, const int64_t* lam,
                        const int64_t* D, const int64_t* o, const int64_t* Lw,
                        int dtype, int64_t batch);
int hdc_prepare_multi(int dims, int n, int op, const int64_t* L,
                      const int64_t* M, const int64_t* m, const int64_t* p,
                      const int64_t* q, const int64_t* D, int dtype,
                      int64_t batch);
int hdc_prepare_real(int dims, const int64_t* L, const int64_t* M,
                     const int64_t* m, const int64_t* p, const int64_t* q,
                     const int64_t* D, int dtype, int64_t batch);

/* Free the cached twiddle tables on every device (call with no work in
 * flight that uses them; later convolution calls need a new preparation). */
int hdc_release_caches(void);

/* ------------------------------------------------- allocation-free call
 * No counterpart in the paper: an addition for callers that cannot allocate
 * device memory while they run (a plugin inside an application that owns
 * the device-memory budget; a real-time loop that cannot take cudaMalloc's
 * implicit synchronisation and unbounded latency).
 *
 * hdc_conv1d_noalloc computes the same 1-D convolution as hdc_conv1d (same
 * parameters and results) but calls no cudaMalloc, cudaFree or allocating
 * library routine, takes no workspace and leaves the twiddle cache alone.
 * Its scratch -- the twiddle tables (q m entries, and m entries in two
 * forms) and the D x batch x m residue workspace, each rounded up to 256
 * bytes -- lives in
 * one fixed device array of HDC_NOALLOC_SCRATCH_BYTES that every GPU loading
 * the library holds until the process exits.
 *  - f, g, h: device pointers (batch x L complex); h may alias neither f nor
 *    g (there is no in-place mode here).
 *  - Only the single-tile route: m <= 2048 (complex<double>) or m <= 4096
 *    (complex<float>).  Sizes whose scratch exceeds the array, or larger m,
 *    return HDC_ERR_UNSUPPORTED_SIZE before anything is launched; other
 *    errors as hdc_conv1d.
 *  - The first call on a device, with that device current, looks up the
 *    array's device address (cudaGetSymbolAddress) and keeps it; make that
 *    first call before any stream capture.  Under CUDA's default lazy
 *    module loading that first call is also when the driver loads the
 *    library's kernels and places the array in device memory (an implicit
 *    allocation and synchronisation by the driver), so make one call per
 *    device before the phase that must not allocate, or set
 *    CUDA_MODULE_LOADING=EAGER so the driver does it when the library is
 *    loaded.
 *  - The fold/unfold twiddles zeta_N^k come from one table of N = q m
 *    entries in both dtypes (the regular complex<float> route splits a table
 *    above 2^16 entries into two smaller ones); every entry is one FP64
 *    sincospi rounded once, so the results agree to rounding.
 *  - All calls share the one array and every call rewrites what it reads,
 *    so nothing from an earlier call leaks into a result; but calls whose
 *    work overlaps on the GPU (other streams, other host threads) race on
 *    the array: order them on one stream or synchronise between them. */
#define HDC_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
int hdc_conv1d_noalloc(const void* f, const void* g, void* h, int64_t L,
                       int64_t M, int64_t m, int64_t p, int64_t q, int64_t D,
                       int dtype, int64_t batch, void* stream);

/* ----------------------------------------------------- parameter search
 * Section 4.2 (A0 grid search, separable per axis).  Candidates of an axis:
 * for every q, the m = 2^a 3^b 5^c 7^d >= m_min that pad M least (the three
 * smallest >= ceil(M/q), the next power of two, the next 3 * 2^k), p and q
 * derived, D = q; kept when the model flops F1 are within max_ratio (>= 1)
 * of the axis minimum; sorted by F1 (an axis with nextgood(M) < m_min uses
 * m_min = nextgood(M)).  Writes up to `cap` entries, the full count to *n. */
int hdc_tune_candidates(int64_t L, int64_t M, int dtype, double max_ratio,
                        int64_t m_min, hdc_tuple* out, int64_t cap, int64_t* n);

/* Largest workspace any candidate combination of the search needs. */
int hdc_tune_workspace_size(int dims, const int64_t* L, const int64_t* M,
                            int dtype, int64_t batch, double max_ratio,
                            int64_t m_min, size_t* bytes);

/* Time candidates on the caller's device buffers (f, g, h: batch x L;
 * workspace of hdc_tune_workspace_size) with `warmup` untimed and `reps`
 * timed runs each (median of CUDA-graph replays with the L2 evicted before
 * each, on a private stream; more replays, up to 41, while the sample holds
 * less than 1 ms; synchronises `stream`).  Axes are searched one at a time,
 * last axis first, the others held at their best so far; the four fastest
 * candidates of an axis and its explicit one are timed twice more,
 * interleaved, and keep the median of three; the three fastest m are then
 * re-timed with D = 1, 2, 4, ... < q; a time within 1 % of the best goes to
 * explicit padding.
 * best[dims] receives the choice; trials (optional, cap records of dims
 * tuples each) every timed configuration, *ntrials their count. */
int hdc_tune_convnd(int dims, const int64_t* L, const int64_t* M, int dtype,
                    int64_t batch, const void* f, const void* g, void* h,
                    void* workspace, size_t ws_bytes, int warmup, int reps,
                    double max_ratio, int64_t m_min, void* stream,
                    hdc_tuple* best, hdc_tuple* trials, int64_t cap,
                    int64_t* ntrials);
int hdc_tune_conv1d(int64_t L, int64_t M, int dtype, int64_t batch,
                    const void* f, const void* g, void* h, void* workspace,
                    size_t ws_bytes, int warmup, int reps, double max_ratio,
                    int64_t m_min, void* stream, hdc_tuple* best,
                    hdc_tuple* trials, int64_t cap, int64_t* ntrials);

/* The same search for unequal lengths (hdc_convnd_unequal, first Lg
 * outputs per axis).  Candidates of an axis: for every qg, the g transform
 * sizes mg that pad M least (as above, mg >= m_min), each with lam = 1 and
 * every lam = 2^a or 3 * 2^a dividing mg whose f size m = mg / lam lies in
 * [Lf / 2, 2 Lf] (f's cost 5 mg log2 m + 8 lam Lf per g residue is least
 * near m = Lf); kept when
 * the model flops
 *   F_u = qg (10 mg log2 mg + 5 lam m log2 m + 6 mg + 8 (Lg + lam Lf + Lg)) + 2 Lg
 * are within max_ratio of the axis minimum, sorted by F_u.  M = NULL (or
 * M[i] <= 0) takes the least alias-free M = Lf + Lg - 1.  hdc_tune_unequal
 * times them on the caller's buffers (f: batch x prod(Lf), g and h:
 * batch x prod(Lg)) like hdc_tune_convnd; with a non-NULL tuning_db it
 * first looks the problem up there and appends what it finds. */
typedef struct hdc_unequal_tuple {
    int64_t m, lam, q, D; /* f size m, g size lam m, g residues qg, per pass */
    double model_flops;   /* F_u of the axis                               */
    double ms;            /* median device time of the whole call, or -1   */
} hdc_unequal_tuple;
int hdc_tune_unequal_candidates(int64_t Lf, int64_t Lg, int64_t M, int dtype,
                                double max_ratio, int64_t m_min,
                                hdc_unequal_tuple* out, int64_t cap,
                                int64_t* n);
int hdc_tune_unequal_workspace_size(int dims, const int64_t* Lf,
                                    const int64_t* Lg, const int64_t* M,
                                    int dtype, int64_t batch, double max_ratio,
                                    int64_t m_min, size_t* bytes);
int hdc_tune_unequal(int dims, const int64_t* Lf, const int64_t* Lg,
                     const int64_t* M, int dtype, int64_t batch, const void* f,
                     const void* g, void* h, void* workspace, size_t ws_bytes,
                     int warmup, int reps, double max_ratio, int64_t m_min,
                     const char* tuning_db, void* stream,
                     hdc_unequal_tuple* best, hdc_unequal_tuple* trials,
                     int64_t cap, int64_t* ntrials);

/* The same search for the multi-convolution of n inputs with operator op
 * (hdc_convnd_multi): the candidates of hdc_tune_candidates for (L, M) per
 * axis (M alias-free for op, else HDC_ERR_ALIAS), timed on the caller's
 * inputs[n] and h. */
int hdc_tune_multi_workspace_size(int dims, int n, int op, const int64_t* L,
                                  const int64_t* M, int dtype, int64_t batch,
                                  double max_ratio, int64_t m_min,
                                  size_t* bytes);
int hdc_tune_multi(int dims, int n, int op, const int64_t* L, const int64_t* M,
                   int dtype, int64_t batch, const void* const* inputs,
                   void* h, void* workspace, size_t ws_bytes, int warmup,
                   int reps, double max_ratio, int64_t m_min, void* stream,
                   hdc_tuple* best, hdc_tuple* trials, int64_t cap,
                   int64_t* ntrials);

/* The same search for hdc_convnd_real on the caller's real buffers f, g,
 * h (batch x prod(L)); workspace from hdc_tune_real_workspace_size. */
int hdc_tune_real_workspace_size(int dims, const int64_t* L, const int64_t* M,
                                 int dtype, int64_t batch, double max_ratio,
                                 int64_t m_min, size_t* bytes);
int hdc_tune_real(int dims, const int64_t* L, const int64_t* M, int dtype,
                  int64_t batch, const void* f, const void* g, void* h,
                  void* workspace, size_t ws_bytes, int warmup, int reps,
                  double max_ratio, int64_t m_min, void* stream,
                  hdc_tuple* best, hdc_tuple* trials, int64_t cap,
                  int64_t* ntrials);

/* Cheap searches (Section 4.3, A1: random search and reuse of a
 * rectangle's parameters; Section 6.3: the height-32 rectangle), same
 * buffers and results as hdc_tune_convnd.
 * hdc_tune_convnd_random: random search; per axis n_samples candidates
 * (<= 0: a quarter of them, at least 3) drawn without replacement with a
 * SplitMix64 stream seeded by `seed`, then the separable search over those.
 * hdc_tune_convnd_proxy: for each axis, the separable search on the
 * rectangle in which every other axis longer than Lproxy is cut to Lproxy
 * points (M = 2 Lproxy - 1), run on prefixes of f, g, h; the axis keeps the
 * rectangle's choice for itself.  The workspace of hdc_tune_workspace_size
 * for the full problem suffices (else HDC_ERR_WORKSPACE). *ntrials: timed
 * configurations in all. */
int hdc_tune_convnd_random(int dims, const int64_t* L, const int64_t* M,
                           int dtype, int64_t batch, const void* f,
                           const void* g, void* h, void* workspace,
                           size_t ws_bytes, int warmup, int reps,
                           double max_ratio, int64_t m_min, int64_t n_samples,
                           uint64_t seed, void* stream, hdc_tuple* best,
                           hdc_tuple* trials, int64_t cap, int64_t* ntrials);
int hdc_tune_convnd_proxy(int dims, const int64_t* L, const int64_t* M,
                          int dtype, int64_t batch, const void* f,
                          const void* g, void* h, void* workspace,
                          size_t ws_bytes, int warmup, int reps,
                          double max_ratio, int64_t m_min, int64_t Lproxy,
                          void* stream, hdc_tuple* best, int64_t* ntrials);

/* ---------------------------------------------------------------- plans
 * A plan fixes (m, p, q, D) per axis for one (dims, L, M, dtype, batch).
 * HDC_TUNE_EXHAUSTIVE looks the problem up in the text database at
 * `tuning_db` (may be NULL) and otherwise runs hdc_tune_convnd on scratch
 * buffers it allocates and frees itself (the one place besides twiddle
 * tables where the library allocates), then appends the result to the
 * database.  HDC_FIXED takes m (and D, may be NULL) from the caller.
 * HDC_PREDICT_MLP reads the network checkpoint at `tuning_db` (written by
 * hdc_mlp_save with HDC_MLP_FEATURES inputs, HDC_MLP_HIDDEN hidden units and
 * hdc_mlp_num_q_classes() + 2 outputs) and runs its inference kernels;
 * HDC_PREDICT_MLP_SEARCH then times, for every axis, the network's three
 * most likely valid classes and the valid neighbouring q classes (one down,
 * one up) of its best two, at most six distinct m (one axis at a time, last
 * first, the others held), on scratch buffers it allocates and frees, and
 * keeps the fastest.  Every mode ends by making the twiddle tables the
 * plan's execution reads (hdc_prepare), so hdc_plan_execute allocates
 * nothing and may be captured in a CUDA graph from its first call. */
int hdc_plan_create(hdc_plan** plan, int dims, const int64_t* L,
                    const int64_t* M, const int64_t* m, const int64_t* D,
                    int dtype, int64_t batch, int mode, const char* tuning_db,
                    void* stream);
/* Per-axis parameters of the plan (arrays of length dims; NULL skips). */
int hdc_plan_params(const hdc_plan* plan, int64_t* m, int64_t* p, int64_t* q,
                    int64_t* D);
/* Device workspace bytes hdc_plan_execute needs (in-place included). */
size_t hdc_plan_workspace(const hdc_plan* plan);
/* Configurations timed on the device while the plan was made (0 for the
 * fixed and explicit modes, a database hit or the top-class prediction). */
int64_t hdc_plan_timed(const hdc_plan* plan);
int hdc_plan_execute(const hdc_plan* plan, const void* f, const void* g,
                     void* h, void* workspace, size_t ws_bytes, void* stream);
int hdc_plan_destroy(hdc_plan* plan);

/* ---------------------------------------------------- batched execution
 * n independent 1-D convolutions of uneven lengths L_i (M_i = 2 L_i - 1,
 * FFT size m_i per convolution, p_i and q_i derived, all residues in one
 * pass) in ONE cooperative persistent launch: blocks claim work items of
 * four phases (column fold+FFT, row transforms, column inverse FFT, unfold)
 * from atomic counters and meet at a grid barrier between phases.  The
 * barrier's spin is bounded; if it runs out, the status word in the
 * workspace becomes HDC_ERR_TIMEOUT and the blocks return.  The launch and
 * the memset that clears its counters may be captured in a CUDA graph.
 * No counterpart in the paper (its method convolves one problem at a time).
 *
 * create: validates every (L_i, 2 L_i - 1, m_i), builds the work lists and
 *   uploads them (library-owned device memory, freed by destroy).
 * execute: f, g, h are DEVICE arrays of n device pointers (each to L_i
 *   complex values); workspace of hdc_batched_workspace() bytes. */
typedef struct hdc_batched hdc_batched;
int hdc_batched_create(hdc_batched** plan, int64_t n, const int64_t* L,
                       const int64_t* m, int dtype);
size_t hdc_batched_workspace(const hdc_batched* plan);
/* per-convolution m, p, q and the split m = m1 m2 (m1 = 0: one row tile) */
int hdc_batched_params(const hdc_batched* plan, int64_t* m, int64_t* p,
                       int64_t* q, int64_t* m1, int64_t* m2);
int hdc_batched_execute(hdc_batched* plan, const void* const* f,
                        const void* const* g, void* const* h, void* workspace,
                        size_t ws_bytes, void* stream);
/* Status word of the last execute in `workspace` (synchronous copy; call
 * after the stream has finished): 0 or HDC_ERR_TIMEOUT. */
int hdc_batched_status(const void* workspace, int* status);
/* Durations (ms, from the GPU's global timer) of the four phases of the last
 * execute in `workspace` (column folds and FFTs, rows, inverse column FFTs,
 * unfolds), each from the grid barrier that opens it to the one that closes
 * it, the last to the end of the last block (synchronous copy; call after
 * the stream has finished). */
int hdc_batched_phase_ms(const void* workspace, double* ms);
/* Barrier limits: spin iterations (about 64 ns each) before giving up, and
 * arrivals the barrier waits for beyond the grid (0 in normal use; a
 * positive value makes every barrier wait for blocks that do not exist,
 * which exercises the timeout path without a fault). */
int hdc_batched_set_barrier(hdc_batched* plan, long long spin_limit,
                            int extra_arrivals);
int hdc_batched_destroy(hdc_batched* plan);
/* Per-size schedules (the grid search of Section 4.2 applied to the batched
 * kernel, with size classes as the separable axes): lengths are grouped by
 * floor(log2 L); a group's schedule is its residue count q (from 1, 2, 3,
 * 4, 5, 6, 8, 10, 12, 16) with a size rule, and every member gets its own
 * m >= ceil((2 L_i - 1) / q): the next 2^a 3^b 5^c 7^d, the next 2^a or
 * 3 2^a (more padding but cheaper radix-2/4/8 transforms), or the next 2^a,
 * 3 2^a or 5 2^a.  The first `max_cands` usable (q, rule) pairs, in that
 * order and without rules that repeat the one before, are timed.  All
 * groups start at q = 1, nextgood (explicit padding); then group by group (largest total length
 * first, the others held) each q is timed on the WHOLE batch with this
 * kernel (`reps` timed runs, median) and the fastest kept.  m_out receives
 * every convolution's m.  f_host, g_host, h_host: HOST arrays of the n
 * device pointers.  Allocates and frees its own scratch; synchronises
 * `stream`.  *ms_out: the time of the final assignment. */
int hdc_batched_tune(int64_t n, const int64_t* L, int dtype,
                     const void* const* f_host, const void* const* g_host,
                     void* const* h_host, int reps, int max_cands,
                     void* stream, int64_t* m_out, double* ms_out);

/* ------------------------------------------------- learned predictor (MLP)
 * A per-axis classifier of the parameters (the paper's Section 5.3 finds
 * classification better than regression; Section 4.2's separability lets
 * each axis be predicted on its own): FP32 MLP n_in -> H -> H -> H -> n_out
 * with ReLU, hand-written forward / backward / Adam kernels, deterministic
 * sums.  Heads: outputs [0, n_q) score the residue-count classes
 * hdc_mlp_q_class(k), outputs [n_q, n_q + 2) score D = q versus D = 1.
 * Parameters: one float vector, per layer W[i][o] (row-major) then b[o].
 * Device memory of the network is library-owned (create/destroy). */
#define HDC_MLP_FEATURES 12
#define HDC_MLP_HIDDEN 64
typedef struct hdc_mlp hdc_mlp;
int hdc_mlp_create(hdc_mlp** net, int n_in, int n_hidden, int n_out);
int hdc_mlp_num_params(const hdc_mlp* net);
/* host <-> device parameter copies (set also clears the Adam state) */
int hdc_mlp_set_params(hdc_mlp* net, const float* host);
int hdc_mlp_get_params(const hdc_mlp* net, float* host);
int hdc_mlp_get_grads(const hdc_mlp* net, float* host);
/* X: device n x n_in; logits: device n x n_out */
int hdc_mlp_forward(hdc_mlp* net, const float* X, int64_t n, float* logits,
                    void* stream);
/* Forward, mean softmax cross-entropy of both heads (labels yq in [0, n_q),
 * yd in {0, 1}; -1 skips a head) into *loss (device float), gradients kept
 * in the network.  X, yq, yd, loss: device pointers. */
int hdc_mlp_loss_grad(hdc_mlp* net, const float* X, const int* yq,
                      const int* yd, int64_t n, int n_q, float* loss,
                      void* stream);
/* One Adam step (bias-corrected) with the stored gradients. */
int hdc_mlp_adam(hdc_mlp* net, float lr, float beta1, float beta2, float eps,
                 void* stream);
/* Checkpoint (parameters, Adam moments, step count) to / from a file. */
int hdc_mlp_save(const hdc_mlp* net, const char* path);
int hdc_mlp_load(hdc_mlp* net, const char* path);
int hdc_mlp_destroy(hdc_mlp* net);
/* Residue-count classes: count, value of class k, nearest class of q. */
int hdc_mlp_num_q_classes(void);
int64_t hdc_mlp_q_class(int k);
int hdc_mlp_q_to_class(int64_t q);
/* HDC_MLP_FEATURES features per axis of a problem (dims x 12 floats): log2 L,
 * M / L, innermost or not, log2 of the inner and outer extents, dims, dtype,
 * log2 of all outputs, and for q = 1..4 the padding of q residues of the
 * smallest good m >= ceil(M / q) (plus 1 where m exceeds an outer axis'
 * column-tile limit). */
int hdc_mlp_axis_features(int dims, const int64_t* L, const int64_t* M,
                          int dtype, int64_t batch, float* out);
/* (m, p, q, D) of one axis from its logits: the most likely residue class
 * whose tuple is valid with m <= max_m (0: no bound), m = nextgood(ceil(M /
 * q)), D from the D head.  rank > 0 skips the `rank` most likely valid
 * classes (the k-th best guess, for searches over the top classes). */
/* Parameters of one axis for the q class with index k
 * (hdc_mlp_q_class(k)): m = nextgood(ceil(M / q_k)), D = 1 if one else q;
 * HDC_ERR_UNSUPPORTED_SIZE when m > max_m (max_m > 0) or the tuple is not
 * valid. */
int hdc_mlp_decode_class(int k, int one, int64_t L, int64_t M, int dtype,
                         int64_t max_m, int64_t* m, int64_t* p, int64_t* q,
                         int64_t* D);
int hdc_mlp_decode_axis(const float* logits, int n_q, int64_t L, int64_t M,
                        int dtype, int64_t max_m, int rank, int64_t* m,
                        int64_t* p, int64_t* q, int64_t* D);

/* ------------------------------------------------------ launch statistics
 * Counting of every kernel launch (always on) and, when enabled, CUDA events
 * recorded on the launch stream around each launch.  Read after the work
 * has completed (synchronise first). */
int hdc_stats_reset(void);
int hdc_stats_timing(int on);
int hdc_stats_kernel_count(void);
const char* hdc_stats_kernel_name(int id);
int64_t hdc_stats_total_launches(void);
/* launches, summed event time (ms), model flops and algorithmic bytes of
 * kernel `id` since the last reset. */
int hdc_stats_get(int id, int64_t* launches, double* ms, double* flops,
                  double* bytes);

/* -------------------------------------------------------- load path, status
 * The strided fold (the column pass of a split axis and of the outer axes
 * of 2-D/3-D) stages its tiles in shared memory with TMA tensor copies when
 * the input meets the copy rules (16-byte aligned base and row strides,
 * at most two fold blocks per tile), else with plain loads; both give the
 * same result.  hdc_set_tma(0) forces the plain loads for later launches,
 * hdc_set_tma(1) (the default) allows the copies.  Not thread-safe against
 * launches in flight on other host threads.
 *
 * A kernel whose wait for a copy runs past about a second records
 * HDC_ERR_TIMEOUT in a device status word instead of waiting on (the
 * launch's output is then not valid).  hdc_device_status stores the word
 * (0 when no kernel gave up) in *status after synchronising with the
 * device's current work, and clears it if `clear` is non-zero. */
int hdc_set_tma(int enable);

/* A 1-D convolution of equal-length inputs with only a few rows (rows x C
 * at most the SM count) whose m-point residue fits a cluster (m = m1 m2 with
 * C dividing both) may run whole on thread-block clusters of C = 2..16
 * blocks: per row one cluster takes every residue from fold to unfold in one
 * launch, its transforms split over the blocks and transposed through
 * distributed shared memory, the outputs written once.  Same results as the
 * other routes.  hdc_set_cluster(mode) for later calls: 0 never, 1 (the
 * default) where it is the faster route (small residues in few passes: in
 * FP64 up to 8192 points with one residue, 4096 with two in one pass, and
 * calls that would otherwise run several passes one after another; in FP32
 * one residue up to 16384 points and multi-pass calls; in both, residues of
 * a power of two up to 4096 points, whose transforms run as warp shuffles,
 * up to four residues), 2 wherever the residue fits; HDC_ERR_PARAM for
 * another mode.  Not thread-safe against
 * calls in flight on other host threads. */
int hdc_set_cluster(int mode);
int hdc_device_status(int* status, int clear);

/* ------------------------------------------------------------ measurement
 * Vector FMA throughput probe: the arithmetic roofline of this path (it runs
 * on the FP64/FP32 pipes, not on tensor cores).  Launches `blocks` x
 * `threads` threads that each run 8 independent FMA chains for `iters`
 * iterations in FP64 (dtype HDC_C128) or FP32 (HDC_C64) on `stream`; `out`
 * is a device buffer of blocks*threads elements of that real type (written
 * only to keep the chains live).  *flops receives 2 * 8 * iters * threads *
 * blocks; the caller times the launch with events.  No paper counterpart:
 * the paper names no hardware. */
int hdc_probe_fma(int dtype, int64_t iters, int blocks, int threads, void* out,
                  void* stream, double* flops);

#ifdef __cplusplus
}
#endif

#endif /* HDC_H */

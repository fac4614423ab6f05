// hdc_noalloc.cu -- a 1-D convolution entry point that allocates no memory.
//
// Some callers cannot allocate device memory once they are running: a plugin
// inside a host application that owns the whole device-memory budget, or a
// real-time loop that cannot accept cudaMalloc's implicit synchronisation
// and unbounded latency.  hdc_conv1d_noalloc serves them: its scratch (the
// twiddle tables and the per-residue workspace of the fused route) lives in
// one file-scope device array of fixed size, so the call itself allocates
// nothing; the caller still passes f, g and h.
//
// The array is a __device__ symbol: every GPU that loads the library holds it
// until the process exits.  Host code cannot use the symbol's name as a
// device address, so the first call on each device (with that device
// current) asks the runtime for the address with cudaGetSymbolAddress and
// keeps it; make that first call before any stream capture.
#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include "hdc.h"
#include "hdc_internal.h"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

constexpr size_t kScratchBytes = HDC_NOALLOC_SCRATCH_BYTES;
static_assert(kScratchBytes % 256 == 0, "scratch size must keep 256-byte alignment");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up once per device).
int scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HDC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return HDC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return HDC_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return HDC_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
int run(const void* f, const void* g, void* h, int64_t L, int64_t m, int64_t p, int64_t q, int64_t D,
        int64_t batch, cudaStream_t st)
{
    using namespace hdc;
    using V = cx<T>;
    if (m > max_row_fft<T>()) return HDC_ERR_UNSUPPORTED_SIZE;
    const int64_t N = q * m;
    const size_t b_twN = align256((size_t)N * sizeof(V));
    const FftPlan fpm = fft_plan<T>(m, rows_r16(m));
    const size_t b_twm = align256((size_t)fpm.tlen * sizeof(V));
    const size_t b_ws = align256((size_t)(D * batch * m) * sizeof(V));
    if (b_twN + 2 * b_twm + b_ws > kScratchBytes) return HDC_ERR_UNSUPPORTED_SIZE;
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != HDC_OK) return rc;
    V* twN = reinterpret_cast<V*>(base);
    V* twm = reinterpret_cast<V*>((unsigned char*)base + b_twN);
    V* twml = reinterpret_cast<V*>((unsigned char*)base + b_twN + b_twm);
    V* ws = reinterpret_cast<V*>((unsigned char*)base + b_twN + 2 * b_twm);
    // every call rewrites the tables and the workspace it reads, so nothing
    // left from an earlier call is used
    if (launch_twiddle_into<T>(twN, N, st) != cudaSuccess) return HDC_ERR_CUDA;
    if (launch_twiddle_fft_into<T>(twm, fpm, false, st) != cudaSuccess) return HDC_ERR_CUDA;
    if (launch_twiddle_fft_into<T>(twml, fpm, true, st) != cudaSuccess) return HDC_ERR_CUDA;
    const double scale = 1.0 / (double)N;
    for (int64_t r0 = 0; r0 < q; r0 += D) {
        const int first = (r0 == 0), last = (r0 + D >= q);
        if (launch_residue_rows_tw<T>((const V*)f, (const V*)g, ws, batch, L, L, m, p, q, r0, D, twN, twm, twml, st) !=
            cudaSuccess)
            return HDC_ERR_CUDA;
        if (launch_unfold_tw<T>((V*)h, ws, batch, L, 1, m, p, q, N, 1, 0, L, r0, D, first, last, scale, twN, st) !=
            cudaSuccess)
            return HDC_ERR_CUDA;
    }
    return HDC_OK;
}

} // namespace

HDC_EXPORT int hdc_conv1d_noalloc(const void* f, const void* g, void* h, int64_t L, int64_t M, int64_t m,
                                  int64_t p, int64_t q, int64_t D, int dtype, int64_t batch, void* stream)
{
    int64_t pr = 0, qr = 0, Dr = 0;
    int rc = hdc_validate_axis(L, M, m, p, q, D, dtype, &pr, &qr, &Dr);
    if (rc != HDC_OK) return rc;
    if (batch < 0) return HDC_ERR_PARAM;
    if (batch == 0) return HDC_OK;
    if (!f || !g || !h || h == f || h == g) return HDC_ERR_PARAM;
    const uintptr_t al = dtype == HDC_C128 ? 15 : 7;
    if (((uintptr_t)f & al) || ((uintptr_t)g & al) || ((uintptr_t)h & al)) return HDC_ERR_PARAM;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == HDC_C128) return run<double>(f, g, h, L, m, pr, qr, Dr, batch, st);
    return run<float>(f, g, h, L, m, pr, qr, Dr, batch, st);
}

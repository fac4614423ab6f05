// hdc_mlp.cu -- the learned parameter predictor: a small FP32 MLP with
// hand-written forward, backward and Adam kernels.
//
// Section 5.3 reports that classifying the parameter beats regressing it;
// the predictor is therefore a classifier applied per axis (Section 4.2's
// separability: each axis' parameters are chosen on their own).  For an axis
// of length L with padded length M it predicts the residue count q (classes
// hdc_mlp_q_class(k)) and whether all residues run in one pass (D = q) or
// one per pass (D = 1); m = nextgood(ceil(M / q)), p = ceil(L / m).
//
// Network: n_in -> H -> H -> H -> n_out, ReLU after the three hidden
// layers, weights W[i][o] row-major and biases per layer in one contiguous
// parameter vector.  Loss: mean over samples of the softmax cross-entropy of
// the q head (the first n_q outputs) plus that of the D head (the next two);
// a label of -1 leaves its head out.  Every sum runs in a fixed order (no
// atomics), so results are deterministic.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "hdc.h"
#include "hdc_internal.h"

#define HDC_EXPORT extern "C" __attribute__((visibility("default")))

namespace {

constexpr int kLayers = 4;

__global__ void k_linear(const float* __restrict__ A, const float* __restrict__ W, const float* __restrict__ b,
                         float* __restrict__ Z, float* __restrict__ Aout, int n, int in, int out)
{
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * out) return;
    const int s = (int)(gid / out), o = (int)(gid - (int64_t)s * out);
    float z = b[o];
    const float* a = A + (int64_t)s * in;
    for (int i = 0; i < in; ++i) z = fmaf(a[i], W[(int64_t)i * out + o], z);
    Z[gid] = z;
    if (Aout) Aout[gid] = z > 0.f ? z : 0.f;
}

// softmax cross-entropy of the q head [0, nq) and the D head [nq, nq + 2)
__global__ void k_ce(const float* __restrict__ logits, const int* __restrict__ yq, const int* __restrict__ yd, int n,
                     int nq, int out, float* __restrict__ dlogits, float* __restrict__ loss)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float* l = logits + (int64_t)s * out;
    float* d = dlogits + (int64_t)s * out;
    float ls = 0.f;
    const float inv = 1.f / (float)n;
    const int lo[2] = { 0, nq }, hi[2] = { nq, nq + 2 };
    const int y[2] = { yq[s], yd[s] };
    for (int k = 0; k < out; ++k) d[k] = 0.f;
    for (int hd = 0; hd < 2; ++hd) {
        if (y[hd] < 0) continue;
        float mx = l[lo[hd]];
        for (int k = lo[hd] + 1; k < hi[hd]; ++k) mx = fmaxf(mx, l[k]);
        float se = 0.f;
        for (int k = lo[hd]; k < hi[hd]; ++k) se += expf(l[k] - mx);
        const float lse = mx + logf(se);
        ls += lse - l[lo[hd] + y[hd]];
        for (int k = lo[hd]; k < hi[hd]; ++k) {
            const float pk = expf(l[k] - lse);
            d[k] = (pk - (k - lo[hd] == y[hd] ? 1.f : 0.f)) * inv;
        }
    }
    loss[s] = ls;
}

__global__ void k_sum(const float* __restrict__ x, int n, float* __restrict__ out, float scale)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += (double)x[i];
    *out = (float)(s * scale);
}

// dZprev[s][i] = (sum_o dZ[s][o] W[i][o]) * (Zprev[s][i] > 0)
__global__ void k_backprop(const float* __restrict__ dZ, const float* __restrict__ W, const float* __restrict__ Zprev,
                           float* __restrict__ dZprev, int n, int in, int out)
{
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= (int64_t)n * in) return;
    const int s = (int)(gid / in), i = (int)(gid - (int64_t)s * in);
    float a = 0.f;
    const float* dz = dZ + (int64_t)s * out;
    const float* w = W + (int64_t)i * out;
    for (int o = 0; o < out; ++o) a = fmaf(dz[o], w[o], a);
    dZprev[gid] = Zprev[gid] > 0.f ? a : 0.f;
}

// dW[i][o] = sum_s A[s][i] dZ[s][o] (i < in); db[o] = sum_s dZ[s][o] (i == in)
__global__ void k_weight_grad(const float* __restrict__ A, const float* __restrict__ dZ, float* __restrict__ dW,
                              float* __restrict__ db, int n, int in, int out)
{
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= (int64_t)(in + 1) * out) return;
    const int i = (int)(gid / out), o = (int)(gid - (int64_t)i * out);
    float g = 0.f;
    if (i < in) {
        for (int s = 0; s < n; ++s) g = fmaf(A[(int64_t)s * in + i], dZ[(int64_t)s * out + o], g);
        dW[(int64_t)i * out + o] = g;
    } else {
        for (int s = 0; s < n; ++s) g += dZ[(int64_t)s * out + o];
        db[o] = g;
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
}

unsigned nblk(int64_t n, int thr) { return (unsigned)((n + thr - 1) / thr); }

} // namespace

struct hdc_mlp {
    int n_in, n_hid, n_out, n_params;
    int dims[kLayers + 1];
    int64_t w_off[kLayers], b_off[kLayers];
    float* params = nullptr;
    float* grads = nullptr;
    float* am = nullptr;
    float* av = nullptr;
    int64_t step = 0;
    // activations for up to `cap` samples: Z_l and A_l per layer, dZ per layer, loss per sample
    float* act = nullptr;
    int64_t cap = 0;
};

namespace {

int ensure_cap(hdc_mlp* net, int64_t n)
{
    if (n <= net->cap) return HDC_OK;
    int64_t per = 0;
    for (int l = 1; l <= kLayers; ++l) per += 3 * (int64_t)net->dims[l];
    per += 1;
    cudaFree(net->act);
    net->act = nullptr;
    net->cap = 0;
    if (cudaMalloc(&net->act, (size_t)(per * n) * sizeof(float)) != cudaSuccess) return HDC_ERR_ALLOC;
    net->cap = n;
    return HDC_OK;
}

// activation views for n samples: Z[l], A[l], dZ[l] (l = 1..4), loss
struct Views {
    float* Z[kLayers + 1];
    float* A[kLayers + 1];
    float* dZ[kLayers + 1];
    float* loss;
};

Views views(hdc_mlp* net)
{
    Views v;
    float* p = net->act;
    for (int l = 1; l <= kLayers; ++l) {
        v.Z[l] = p; p += net->cap * net->dims[l];
        v.A[l] = p; p += net->cap * net->dims[l];
        v.dZ[l] = p; p += net->cap * net->dims[l];
    }
    v.loss = p;
    v.Z[0] = v.A[0] = v.dZ[0] = nullptr;
    return v;
}

int forward(hdc_mlp* net, const float* X, int64_t n, cudaStream_t st, Views& v)
{
    const float* a = X;
    for (int l = 1; l <= kLayers; ++l) {
        const int in = net->dims[l - 1], out = net->dims[l];
        float* aout = l < kLayers ? v.A[l] : nullptr;
        k_linear<<<nblk(n * out, 128), 128, 0, st>>>(a, net->params + net->w_off[l - 1], net->params + net->b_off[l - 1],
                                                      v.Z[l], aout, (int)n, in, out);
        a = v.A[l];
    }
    return cudaGetLastError() == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}

} // namespace

HDC_EXPORT int hdc_mlp_create(hdc_mlp** out, int n_in, int n_hidden, int n_out)
{
    if (!out || n_in < 1 || n_hidden < 1 || n_out < 3) return HDC_ERR_PARAM;
    hdc_mlp* net = new (std::nothrow) hdc_mlp;
    if (!net) return HDC_ERR_ALLOC;
    net->n_in = n_in;
    net->n_hid = n_hidden;
    net->n_out = n_out;
    net->dims[0] = n_in;
    net->dims[1] = net->dims[2] = net->dims[3] = n_hidden;
    net->dims[4] = n_out;
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        net->w_off[l] = off;
        off += (int64_t)net->dims[l] * net->dims[l + 1];
        net->b_off[l] = off;
        off += net->dims[l + 1];
    }
    net->n_params = (int)off;
    const size_t b = (size_t)off * sizeof(float);
    if (cudaMalloc(&net->params, b) != cudaSuccess || cudaMalloc(&net->grads, b) != cudaSuccess ||
        cudaMalloc(&net->am, b) != cudaSuccess || cudaMalloc(&net->av, b) != cudaSuccess) {
        cudaFree(net->params); cudaFree(net->grads); cudaFree(net->am); cudaFree(net->av);
        delete net;
        return HDC_ERR_ALLOC;
    }
    cudaMemset(net->params, 0, b);
    cudaMemset(net->grads, 0, b);
    cudaMemset(net->am, 0, b);
    cudaMemset(net->av, 0, b);
    *out = net;
    return HDC_OK;
}

HDC_EXPORT int hdc_mlp_num_params(const hdc_mlp* net) { return net ? net->n_params : 0; }

HDC_EXPORT int hdc_mlp_set_params(hdc_mlp* net, const float* host)
{
    if (!net || !host) return HDC_ERR_PARAM;
    const size_t b = (size_t)net->n_params * sizeof(float);
    if (cudaMemcpy(net->params, host, b, cudaMemcpyHostToDevice) != cudaSuccess) return HDC_ERR_CUDA;
    cudaMemset(net->am, 0, b);
    cudaMemset(net->av, 0, b);
    net->step = 0;
    return HDC_OK;
}

HDC_EXPORT int hdc_mlp_get_params(const hdc_mlp* net, float* host)
{
    if (!net || !host) return HDC_ERR_PARAM;
    return cudaMemcpy(host, net->params, (size_t)net->n_params * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? HDC_OK
               : HDC_ERR_CUDA;
}

HDC_EXPORT int hdc_mlp_get_grads(const hdc_mlp* net, float* host)
{
    if (!net || !host) return HDC_ERR_PARAM;
    return cudaMemcpy(host, net->grads, (size_t)net->n_params * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? HDC_OK
               : HDC_ERR_CUDA;
}

HDC_EXPORT int hdc_mlp_forward(hdc_mlp* net, const float* X, int64_t n, float* logits, void* stream)
{
    if (!net || !X || !logits || n < 1) return HDC_ERR_PARAM;
    int rc = ensure_cap(net, n);
    if (rc != HDC_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Views v = views(net);
    rc = forward(net, X, n, st, v);
    if (rc != HDC_OK) return rc;
    return cudaMemcpyAsync(logits, v.Z[kLayers], (size_t)(n * net->n_out) * sizeof(float), cudaMemcpyDeviceToDevice,
                           st) == cudaSuccess
               ? HDC_OK
               : HDC_ERR_CUDA;
}

HDC_EXPORT int hdc_mlp_loss_grad(hdc_mlp* net, const float* X, const int* yq, const int* yd, int64_t n, int n_q,
                                 float* loss, void* stream)
{
    if (!net || !X || !yq || !yd || !loss || n < 1 || n_q < 1 || n_q + 2 > net->n_out) return HDC_ERR_PARAM;
    int rc = ensure_cap(net, n);
    if (rc != HDC_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Views v = views(net);
    rc = forward(net, X, n, st, v);
    if (rc != HDC_OK) return rc;
    k_ce<<<nblk(n, 128), 128, 0, st>>>(v.Z[kLayers], yq, yd, (int)n, n_q, net->n_out, v.dZ[kLayers], v.loss);
    k_sum<<<1, 1, 0, st>>>(v.loss, (int)n, loss, 1.f / (float)n);
    for (int l = kLayers; l >= 1; --l) {
        const int in = net->dims[l - 1], out = net->dims[l];
        const float* Aprev = l > 1 ? v.A[l - 1] : X;
        k_weight_grad<<<nblk((int64_t)(in + 1) * out, 128), 128, 0, st>>>(
            Aprev, v.dZ[l], net->grads + net->w_off[l - 1], net->grads + net->b_off[l - 1], (int)n, in, out);
        if (l > 1)
            k_backprop<<<nblk(n * in, 128), 128, 0, st>>>(v.dZ[l], net->params + net->w_off[l - 1], v.Z[l - 1],
                                                           v.dZ[l - 1], (int)n, in, out);
    }
    return cudaGetLastError() == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}

HDC_EXPORT int hdc_mlp_adam(hdc_mlp* net, float lr, float beta1, float beta2, float eps, void* stream)
{
    if (!net || lr <= 0.f) return HDC_ERR_PARAM;
    net->step += 1;
    const float bc1 = 1.f - powf(beta1, (float)net->step);
    const float bc2 = 1.f - powf(beta2, (float)net->step);
    k_adam<<<nblk(net->n_params, 256), 256, 0, (cudaStream_t)stream>>>(net->params, net->grads, net->am, net->av,
                                                                       net->n_params, lr, beta1, beta2, eps, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? HDC_OK : HDC_ERR_CUDA;
}

// Checkpoint: magic, sizes, step, then params, Adam m and v (float32, host order).
HDC_EXPORT int hdc_mlp_save(const hdc_mlp* net, const char* path)
{
    if (!net || !path) return HDC_ERR_PARAM;
    std::vector<float> buf((size_t)net->n_params * 3);
    const size_t b = (size_t)net->n_params * sizeof(float);
    if (cudaMemcpy(buf.data(), net->params, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf.data() + net->n_params, net->am, b, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf.data() + 2 * (size_t)net->n_params, net->av, b, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HDC_ERR_CUDA;
    FILE* fp = fopen(path, "wb");
    if (!fp) return HDC_ERR_PARAM;
    const int32_t hdr[5] = { 0x48444d4c, net->n_in, net->n_hid, net->n_out, net->n_params };
    const int64_t step = net->step;
    bool ok = fwrite(hdr, sizeof hdr, 1, fp) == 1 && fwrite(&step, sizeof step, 1, fp) == 1 &&
              fwrite(buf.data(), sizeof(float), buf.size(), fp) == buf.size();
    ok = (fclose(fp) == 0) && ok;
    return ok ? HDC_OK : HDC_ERR_PARAM;
}

HDC_EXPORT int hdc_mlp_load(hdc_mlp* net, const char* path)
{
    if (!net || !path) return HDC_ERR_PARAM;
    FILE* fp = fopen(path, "rb");
    if (!fp) return HDC_ERR_PARAM;
    int32_t hdr[5];
    int64_t step = 0;
    std::vector<float> buf((size_t)net->n_params * 3);
    bool ok = fread(hdr, sizeof hdr, 1, fp) == 1 && hdr[0] == 0x48444d4c && hdr[1] == net->n_in &&
              hdr[2] == net->n_hid && hdr[3] == net->n_out && hdr[4] == net->n_params &&
              fread(&step, sizeof step, 1, fp) == 1 && fread(buf.data(), sizeof(float), buf.size(), fp) == buf.size();
    fclose(fp);
    if (!ok) return HDC_ERR_PARAM;
    const size_t b = (size_t)net->n_params * sizeof(float);
    if (cudaMemcpy(net->params, buf.data(), b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(net->am, buf.data() + net->n_params, b, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(net->av, buf.data() + 2 * (size_t)net->n_params, b, cudaMemcpyHostToDevice) != cudaSuccess)
        return HDC_ERR_CUDA;
    net->step = step;
    return HDC_OK;
}

HDC_EXPORT int hdc_mlp_destroy(hdc_mlp* net)
{
    if (!net) return HDC_OK;
    cudaFree(net->params);
    cudaFree(net->grads);
    cudaFree(net->am);
    cudaFree(net->av);
    cudaFree(net->act);
    delete net;
    return HDC_OK;
}

// ------------------------------------------------- predictor glue (host)

namespace {
const int64_t kQClasses[] = { 1, 2, 3, 4, 5, 6, 8, 12 };
constexpr int kNQ = 8;
} // namespace

HDC_EXPORT int hdc_mlp_num_q_classes(void) { return kNQ; }

HDC_EXPORT int64_t hdc_mlp_q_class(int k) { return (k >= 0 && k < kNQ) ? kQClasses[k] : -1; }

// Class of a residue count: the nearest class in log scale.
HDC_EXPORT int hdc_mlp_q_to_class(int64_t q)
{
    if (q < 1) return -1;
    int best = 0;
    double bd = 1e300;
    for (int k = 0; k < kNQ; ++k) {
        const double d = std::fabs(std::log((double)q) - std::log((double)kQClasses[k]));
        if (d < bd) { bd = d; best = k; }
    }
    return best;
}

// Per-axis features (HDC_MLP_FEATURES = 12 per axis): log2 L / 24,
// M / L - 2, 1 if innermost, log2 of the inner column count / 24, log2 of
// the rows above (outer extents times batch) / 24, dims / 3, 1 for FP64,
// log2 of all outputs / 24, then for q = 1, 2, 3, 4 the padding that q
// residues of the smallest good size m >= ceil(M / q) add,
// 4 log2(q m / M) -- a scale-free description of which residue counts pad
// M well, which carries over from short training axes to long ones -- with
// 1 added when that m exceeds the column-tile limit of an axis that has
// inner axes (the tuple is then not available there).
HDC_EXPORT int hdc_mlp_axis_features(int dims, const int64_t* L, const int64_t* M, int dtype, int64_t batch,
                                     float* out)
{
    if (dims < 1 || dims > HDC_MAX_DIMS || !L || !M || !out || batch < 1) return HDC_ERR_PARAM;
    double total = (double)batch;
    for (int i = 0; i < dims; ++i) {
        if (L[i] < 1 || M[i] < 1) return HDC_ERR_PARAM;
        total *= (double)L[i];
    }
    const int64_t outer_lim = hdc_max_outer_fft_size(dtype);
    for (int i = 0; i < dims; ++i) {
        double inner = 1.0, outer = (double)batch;
        for (int j = i + 1; j < dims; ++j) inner *= (double)L[j];
        for (int j = 0; j < i; ++j) outer *= (double)L[j];
        float* f = out + (int64_t)i * HDC_MLP_FEATURES;
        f[0] = (float)(std::log2((double)L[i]) / 24.0);
        f[1] = (float)((double)M[i] / (double)L[i] - 2.0);
        f[2] = i == dims - 1 ? 1.f : 0.f;
        f[3] = (float)(std::log2(inner) / 24.0);
        f[4] = (float)(std::log2(outer) / 24.0);
        f[5] = (float)dims / 3.f;
        f[6] = dtype == HDC_C128 ? 1.f : 0.f;
        f[7] = (float)(std::log2(total) / 24.0);
        for (int q = 1; q <= 4; ++q) {
            const int64_t m = hdc_next_good_size((M[i] + q - 1) / q);
            double v = m > 0 ? 4.0 * std::log2((double)q * (double)m / (double)M[i]) : 4.0;
            if (i < dims - 1 && m > outer_lim) v += 1.0;
            f[7 + q] = (float)v;
        }
    }
    return HDC_OK;
}

// Parameters of one axis for q class k (m = nextgood(ceil(M / q_k)), D = 1
// if one, else q), or an error if that tuple is not valid (m above max_m
// when max_m > 0, or rejected by hdc_validate_axis).
HDC_EXPORT int hdc_mlp_decode_class(int k, int one, int64_t L, int64_t M, int dtype, int64_t max_m, int64_t* m,
                                    int64_t* p, int64_t* q, int64_t* D)
{
    if (k < 0 || k >= kNQ || !m || !p || !q || !D) return HDC_ERR_PARAM;
    const int64_t qc = kQClasses[k];
    const int64_t mm = hdc_next_good_size((M + qc - 1) / qc);
    if (mm < 1 || (max_m > 0 && mm > max_m)) return HDC_ERR_UNSUPPORTED_SIZE;
    int64_t pp = 0, qq = 0, DD = 0;
    const int rc = hdc_validate_axis(L, M, mm, 0, 0, one ? 1 : 0, dtype, &pp, &qq, &DD);
    if (rc != HDC_OK) return rc;
    *m = mm;
    *p = pp;
    *q = qq;
    *D = DD;
    return HDC_OK;
}

// Parameters of one axis from its n_q + 2 logits.
HDC_EXPORT int hdc_mlp_decode_axis(const float* logits, int n_q, int64_t L, int64_t M, int dtype, int64_t max_m,
                                   int rank, int64_t* m, int64_t* p, int64_t* q, int64_t* D)
{
    if (!logits || n_q != kNQ || !m || !p || !q || !D || rank < 0) return HDC_ERR_PARAM;
    // classes in decreasing score; the rank-th one whose tuple is valid
    std::vector<int> order(kNQ);
    for (int k = 0; k < kNQ; ++k) order[k] = k;
    for (int a = 0; a < kNQ; ++a)
        for (int b = a + 1; b < kNQ; ++b)
            if (logits[order[b]] > logits[order[a]]) std::swap(order[a], order[b]);
    const bool one = logits[kNQ + 1] > logits[kNQ];
    int seen = 0;
    for (int k : order) {
        int64_t mm = 0, pp = 0, qq = 0, DD = 0;
        if (hdc_mlp_decode_class(k, one, L, M, dtype, max_m, &mm, &pp, &qq, &DD) != HDC_OK) continue;
        if (seen++ < rank) continue;
        *m = mm;
        *p = pp;
        *q = qq;
        *D = DD;
        return HDC_OK;
    }
    return HDC_ERR_UNSUPPORTED_SIZE;
}

// Multilayer perceptron used as a learned surrogate of the loop k-sums: training and inference kernels.
//
// Architecture: n_in -> [width, GELU] x depth -> n_out (linear output).  Weights are BF16 and every
// product accumulates in FP32.  Training passes also round the activations to BF16; FP32 master
// weights receive the Adam update and are rounded to BF16 after each step (mixed-precision training).
// Inference keeps the activations in FP32, so the network is a smooth function of its inputs (BF16
// inputs and activations would make it a staircase in log T that an adaptive integrator resolves with
// ever smaller steps).  Loss: mean squared error.
// Kernels: the GEMMs on the tensor cores (k_mlp_tc.cu: BF16 x BF16 for training, FP32 activations split into
// TF32 parts x BF16 weights for inference, FP32 accumulation, fixed summation order), GELU forward/backward, the
// loss gradient, bias gradients as fixed-order column sums, and Adam.  Nothing here is part of the paper: it
// serves the surrogate of the loops.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "tufrg_internal.cuh"

struct tufrg_mlp {
    int n_in = 0, width = 0, depth = 0, n_out = 0;
    int n_layers = 0;                      // depth + 1 linear layers
    std::vector<int> din, dout;            // per layer
    std::vector<size_t> woff, boff;        // offsets in the flat parameter vector
    size_t n_params = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    float *d_w = nullptr;                  // FP32 master parameters (flat)
    __nv_bfloat16 *d_w16 = nullptr;        // BF16 copy used by the kernels
    float *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;   // gradient, Adam moments
    int adam_t = 0;
    int cap = 0;                           // batch capacity of the activation buffers
    std::vector<float *> Z;                // [layer] pre-activations, FP32 [cap][dout]
    std::vector<__nv_bfloat16 *> H;        // [layer + 1] layer inputs, BF16 [cap][din]; H[0] = input
    float *dA = nullptr, *dA2 = nullptr;   // FP32 upstream gradients [cap][max width]
    __nv_bfloat16 *dZ16 = nullptr;         // BF16 copy of dZ
    float *dZ = nullptr;                   // FP32 dZ
    float *loss = nullptr;                 // [1]
    void *ws = nullptr;                    // packed GEMM operands (tensor cores)
    size_t ws_bytes = 0;
    int *d_err = nullptr;                  // raised when a bounded device wait of a GEMM gave up
};

namespace tufrg {
namespace {

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x)
{
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__global__ void to_bf16_kernel(const float *x, __nv_bfloat16 *y, size_t n, const int *skip = nullptr)
{
    if (skip && *skip) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

__device__ __forceinline__ void st_act(__nv_bfloat16 *p, float v) { *p = __float2bfloat16(v); }
__device__ __forceinline__ void st_act(float *p, float v) { *p = v; }

// H = GELU(Z); H may alias Z (FP32 inference, in place)
template <typename TH>
__global__ void gelu_fwd_kernel(const float *Z, TH *H, size_t n, const int *skip)
{
    if (skip && *skip) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        st_act(H + i, gelu(Z[i]));
}

// dZ = dA * gelu'(Z) (hidden layers) or dZ = dA (output layer); FP32 and BF16 copies
__global__ void act_bwd_kernel(const float *dA, const float *Z, int hidden, float *dZ, __nv_bfloat16 *dZ16, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float g = hidden ? dA[i] * gelu_d(Z[i]) : dA[i];
        dZ[i] = g;
        dZ16[i] = __float2bfloat16(g);
    }
}

// dY = 2 (Y - T) / n, and the loss sum((Y - T)^2) / n by a fixed-order block reduction (one block)
__global__ void mse_kernel(const float *Y, const float *T, float *dY, size_t n, float *loss)
{
    __shared__ double sh[256];
    double s = 0.0;
    const float inv = 1.f / (float)n;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d * inv;
        s += (double)d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(sh[0] / (double)n);
}

// db[c] = sum_r dZ[r][c] in row order
__global__ void colsum_kernel(const float *dZ, int rows, int cols, float *db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; r++) s += dZ[(size_t)r * cols + c];
    db[c] = s;
}

__global__ void adam_kernel(float *w, const float *g, float *m, float *v, __nv_bfloat16 *w16, size_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        w16[i] = __float2bfloat16(wi);
    }
}

int gsz(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

tufrg_status mfail(tufrg_mlp *n, tufrg_status st, const std::string &msg)
{
    if (n) n->err = msg;
    (void)cudaGetLastError();   // leave no failed call's error pending for the caller's next launch check
    return st;
}

// a host allocation that failed inside an entry point becomes TUFRG_ENOMEM instead of crossing the C boundary
tufrg_status mlp_host_alloc_fail(tufrg_mlp *n, const std::exception &ex) noexcept
{
    if (n) {
        try {
            n->err = std::string("host allocation failed: ") + ex.what();
        } catch (...) {
            n->err.clear();
        }
    }
    return TUFRG_ENOMEM;
}

#define MK(expr, where)                                                                           \
    do {                                                                                          \
        cudaError_t _e = (expr);                                                                  \
        if (_e != cudaSuccess)                                                                    \
            return mfail(n, _e == cudaErrorMemoryAllocation ? TUFRG_ENOMEM : TUFRG_ECUDA,         \
                         std::string(where) + ": " + cudaGetErrorString(_e));                     \
    } while (0)

// C = op(A) op(B) (+ bias) on the tensor cores with the network's operand scratch
template <typename TA>
cudaError_t gemm(tufrg_mlp *n, cudaStream_t s, const TA *A, int lda, int ta, const __nv_bfloat16 *B, int ldb, int tb,
                 float *C, int ldc, int M, int N, int K, const float *bias, const int *skip = nullptr)
{
    if (mlp_tc_scratch_bytes(M, N, K) > n->ws_bytes) return cudaErrorInvalidValue;   // sized by ensure_capacity
    return mlp_gemm_tc<TA>(s, A, lda, ta, B, ldb, tb, C, ldc, M, N, K, bias, skip, n->ws, n->d_err);
}

tufrg_status ensure_capacity(tufrg_mlp *n, int batch)
{
    if (batch <= n->cap) return TUFRG_OK;
    for (auto p : n->Z) cudaFree(p);
    for (auto p : n->H) cudaFree(p);
    cudaFree(n->dA); cudaFree(n->dA2); cudaFree(n->dZ16); cudaFree(n->dZ);
    n->Z.assign(n->n_layers, nullptr);
    n->H.assign(n->n_layers + 1, nullptr);
    int wmax = n->n_in;
    for (int l = 0; l < n->n_layers; l++) wmax = std::max(wmax, std::max(n->din[l], n->dout[l]));
    for (int l = 0; l < n->n_layers; l++) MK(cudaMalloc(&n->Z[l], sizeof(float) * (size_t)batch * n->dout[l]), "cudaMalloc activations");
    for (int l = 0; l <= n->n_layers; l++) {
        const int w = l < n->n_layers ? n->din[l] : n->n_out;
        MK(cudaMalloc(&n->H[l], sizeof(__nv_bfloat16) * (size_t)batch * w), "cudaMalloc activations");
    }
    MK(cudaMalloc(&n->dA, sizeof(float) * (size_t)batch * wmax), "cudaMalloc gradients");
    MK(cudaMalloc(&n->dA2, sizeof(float) * (size_t)batch * wmax), "cudaMalloc gradients");
    MK(cudaMalloc(&n->dZ, sizeof(float) * (size_t)batch * wmax), "cudaMalloc gradients");
    MK(cudaMalloc(&n->dZ16, sizeof(__nv_bfloat16) * (size_t)batch * wmax), "cudaMalloc gradients");
    // operand scratch of the largest GEMM: the forward (batch x dout x din), weight-gradient (din x dout x batch)
    // and input-gradient (batch x din x dout) products of every layer
    size_t ws = 0;
    for (int l = 0; l < n->n_layers; l++) {
        ws = std::max(ws, mlp_tc_scratch_bytes(batch, n->dout[l], n->din[l]));
        ws = std::max(ws, mlp_tc_scratch_bytes(n->din[l], n->dout[l], batch));
        ws = std::max(ws, mlp_tc_scratch_bytes(batch, n->din[l], n->dout[l]));
    }
    if (ws > n->ws_bytes) {
        cudaFree(n->ws);
        n->ws = nullptr;
        MK(cudaMalloc(&n->ws, ws), "cudaMalloc GEMM operands");
        n->ws_bytes = ws;
    }
    n->cap = batch;
    return TUFRG_OK;
}

// Training forward pass (BF16 activations); Y (FP32 [batch][n_out]) receives the output; keeps the
// hidden pre-activations Z and the layer inputs H for the backward pass (the output layer is linear,
// so its Z is never needed).
tufrg_status forward(tufrg_mlp *n, const float *X, int batch, float *Y)
{
    tufrg_status st = ensure_capacity(n, batch);
    if (st != TUFRG_OK) return st;
    cudaStream_t s = n->stream;
    to_bf16_kernel<<<gsz((size_t)batch * n->n_in), 256, 0, s>>>(X, n->H[0], (size_t)batch * n->n_in);
    MK(cudaGetLastError(), "convert input");
    for (int l = 0; l < n->n_layers; l++) {
        const bool last = l == n->n_layers - 1;
        float *out = last ? Y : n->Z[l];
        MK(gemm(n, s, n->H[l], n->din[l], 0, n->d_w16 + n->woff[l], n->dout[l], 0, out, n->dout[l], batch, n->dout[l],
                n->din[l], n->d_w + n->boff[l]), "layer GEMM");
        if (!last) {
            gelu_fwd_kernel<<<gsz((size_t)batch * n->dout[l]), 256, 0, s>>>(n->Z[l], n->H[l + 1], (size_t)batch * n->dout[l],
                                                                            (const int *)nullptr);
            MK(cudaGetLastError(), "GELU");
        }
    }
    return TUFRG_OK;
}

// Inference forward pass: BF16 weights, FP32 input and activations (GELU in place on Z).  With
// skip != NULL every kernel returns at once while *skip != 0 (device-side decision, graph-capturable).
tufrg_status infer(tufrg_mlp *n, const float *X, int batch, float *Y, const int *skip)
{
    tufrg_status st = ensure_capacity(n, batch);
    if (st != TUFRG_OK) return st;
    cudaStream_t s = n->stream;
    const float *in = X;
    for (int l = 0; l < n->n_layers; l++) {
        const bool last = l == n->n_layers - 1;
        float *out = last ? Y : n->Z[l];
        MK(gemm(n, s, in, n->din[l], 0, n->d_w16 + n->woff[l], n->dout[l], 0, out, n->dout[l], batch, n->dout[l], n->din[l],
                n->d_w + n->boff[l], skip), "layer GEMM");
        if (!last) {
            gelu_fwd_kernel<<<gsz((size_t)batch * n->dout[l]), 256, 0, s>>>(n->Z[l], n->Z[l], (size_t)batch * n->dout[l],
                                                                            skip);
            MK(cudaGetLastError(), "GELU");
            in = n->Z[l];
        }
    }
    return TUFRG_OK;
}

// backward pass from dY = dLoss/dY into the flat gradient g
tufrg_status backward(tufrg_mlp *n, int batch, const float *dY, float *g)
{
    cudaStream_t s = n->stream;
    const float *up = dY;
    for (int l = n->n_layers - 1; l >= 0; l--) {
        const size_t cnt = (size_t)batch * n->dout[l];
        const bool hidden = l < n->n_layers - 1;
        act_bwd_kernel<<<gsz(cnt), 256, 0, s>>>(up, n->Z[l], hidden ? 1 : 0, n->dZ, n->dZ16, cnt);
        MK(cudaGetLastError(), "activation backward");
        // dW = H^T dZ  (din x dout), db = column sums of dZ
        MK(gemm(n, s, n->H[l], n->din[l], 1, n->dZ16, n->dout[l], 0, g + n->woff[l], n->dout[l], n->din[l], n->dout[l],
                batch, nullptr), "weight gradient");
        colsum_kernel<<<(n->dout[l] + 127) / 128, 128, 0, s>>>(n->dZ, batch, n->dout[l], g + n->boff[l]);
        MK(cudaGetLastError(), "bias gradient");
        if (l > 0) {
            // dH = dZ W^T  (batch x din)
            float *dst = (up == n->dA) ? n->dA2 : n->dA;
            MK(gemm(n, s, n->dZ16, n->dout[l], 0, n->d_w16 + n->woff[l], n->dout[l], 1, dst, n->din[l], batch, n->din[l],
                    n->dout[l], nullptr), "input gradient");
            up = dst;
        }
    }
    return TUFRG_OK;
}

}  // namespace
}  // namespace tufrg

using namespace tufrg;

extern "C" {

tufrg_status tufrg_mlp_create(int n_in, int width, int depth, int n_out, unsigned long long seed, void *cuda_stream,
                              tufrg_mlp **out)
try {
    if (!out) return TUFRG_EINVAL;
    *out = nullptr;
    if (n_in < 1 || width < 1 || depth < 1 || n_out < 1 || n_in > 4096 || width > 4096 || n_out > 65536) return TUFRG_EINVAL;
    tufrg_mlp *n = new (std::nothrow) tufrg_mlp();
    if (!n) return TUFRG_ENOMEM;
    *out = n;
    n->n_in = n_in; n->width = width; n->depth = depth; n->n_out = n_out;
    n->n_layers = depth + 1;
    n->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    for (int l = 0; l < n->n_layers; l++) {
        n->din.push_back(l == 0 ? n_in : width);
        n->dout.push_back(l == n->n_layers - 1 ? n_out : width);
    }
    size_t off = 0;
    for (int l = 0; l < n->n_layers; l++) {
        n->woff.push_back(off);
        off += (size_t)n->din[l] * n->dout[l];
        n->boff.push_back(off);
        off += n->dout[l];
    }
    n->n_params = off;
    // He-style uniform initialisation from the seed (host), zero biases
    std::vector<float> w(off, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < n->n_layers; l++) {
        const float a = std::sqrt(6.f / (float)n->din[l]) * (l == n->n_layers - 1 ? 0.5f : 1.f);
        std::uniform_real_distribution<float> U(-a, a);
        for (size_t i = 0; i < (size_t)n->din[l] * n->dout[l]; i++) w[n->woff[l] + i] = U(rng);
    }
    MK(cudaMalloc(&n->d_w, sizeof(float) * off), "cudaMalloc parameters");
    MK(cudaMalloc(&n->d_w16, sizeof(__nv_bfloat16) * off), "cudaMalloc parameters");
    MK(cudaMalloc(&n->d_g, sizeof(float) * off), "cudaMalloc gradients");
    MK(cudaMalloc(&n->d_m, sizeof(float) * off), "cudaMalloc moments");
    MK(cudaMalloc(&n->d_v, sizeof(float) * off), "cudaMalloc moments");
    MK(cudaMalloc(&n->loss, sizeof(float)), "cudaMalloc loss");
    MK(cudaMalloc(&n->d_err, sizeof(int)), "cudaMalloc error flag");
    MK(cudaMemsetAsync(n->d_err, 0, sizeof(int), n->stream), "zero");
    MK(cudaMemcpyAsync(n->d_w, w.data(), sizeof(float) * off, cudaMemcpyHostToDevice, n->stream), "copy parameters");
    MK(cudaMemsetAsync(n->d_m, 0, sizeof(float) * off, n->stream), "zero");
    MK(cudaMemsetAsync(n->d_v, 0, sizeof(float) * off, n->stream), "zero");
    to_bf16_kernel<<<gsz(off), 256, 0, n->stream>>>(n->d_w, n->d_w16, off);
    MK(cudaGetLastError(), "convert parameters");
    MK(cudaStreamSynchronize(n->stream), "sync");
    return TUFRG_OK;
} catch (const std::exception &ex) {
    return mlp_host_alloc_fail(out ? *out : nullptr, ex);
}

void tufrg_mlp_free(tufrg_mlp *n)
{
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    for (auto p : n->Z) cudaFree(p);
    for (auto p : n->H) cudaFree(p);
    void *ptrs[] = {n->d_w, n->d_w16, n->d_g, n->d_m, n->d_v, n->loss, n->dA, n->dA2, n->dZ16, n->dZ, n->ws, n->d_err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete n;
}

const char *tufrg_mlp_last_error(const tufrg_mlp *n) { return n ? n->err.c_str() : "network handle is NULL"; }

long long tufrg_mlp_num_params(const tufrg_mlp *n) { return n ? (long long)n->n_params : -1; }

tufrg_status tufrg_mlp_get_params(tufrg_mlp *n, float *h_params)
{
    if (!n || !h_params) return TUFRG_EINVAL;
    MK(cudaMemcpyAsync(h_params, n->d_w, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost, n->stream), "copy");
    MK(cudaStreamSynchronize(n->stream), "sync");
    return TUFRG_OK;
}

tufrg_status tufrg_mlp_set_params(tufrg_mlp *n, const float *h_params)
{
    if (!n || !h_params) return TUFRG_EINVAL;
    MK(cudaMemcpyAsync(n->d_w, h_params, sizeof(float) * n->n_params, cudaMemcpyHostToDevice, n->stream), "copy");
    to_bf16_kernel<<<gsz(n->n_params), 256, 0, n->stream>>>(n->d_w, n->d_w16, n->n_params);
    MK(cudaGetLastError(), "convert parameters");
    MK(cudaStreamSynchronize(n->stream), "sync");
    n->adam_t = 0;
    MK(cudaMemsetAsync(n->d_m, 0, sizeof(float) * n->n_params, n->stream), "zero");
    MK(cudaMemsetAsync(n->d_v, 0, sizeof(float) * n->n_params, n->stream), "zero");
    return TUFRG_OK;
}

tufrg_status tufrg_mlp_forward(tufrg_mlp *n, const float *d_X, int batch, float *d_Y)
{
    if (!n || !d_X || !d_Y || batch < 1) return TUFRG_EINVAL;
    return infer(n, d_X, batch, d_Y, nullptr);
}

tufrg_status tufrg_mlp_gradients(tufrg_mlp *n, const float *d_X, const float *d_T, int batch, float *d_grad, float *h_loss)
{
    if (!n || !d_X || !d_T || !d_grad || batch < 1) return TUFRG_EINVAL;
    tufrg_status st = ensure_capacity(n, batch);
    if (st != TUFRG_OK) return st;
    float *Y = n->dA2;   // output buffer reused (overwritten by the backward pass only after dY is formed)
    float *dY = n->dA;
    // the output and its gradient need [batch][n_out]; dA/dA2 are sized for max(width, n_out)
    if ((st = forward(n, d_X, batch, Y)) != TUFRG_OK) return st;
    const size_t cnt = (size_t)batch * n->n_out;
    mse_kernel<<<1, 256, 0, n->stream>>>(Y, d_T, dY, cnt, n->loss);
    MK(cudaGetLastError(), "loss");
    if ((st = backward(n, batch, dY, d_grad)) != TUFRG_OK) return st;
    if (h_loss) {
        int e = 0;
        MK(cudaMemcpyAsync(h_loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream), "copy loss");
        MK(cudaMemcpyAsync(&e, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream), "copy error flag");
        MK(cudaStreamSynchronize(n->stream), "sync");
        if (e) return mfail(n, TUFRG_ETIMEOUT, "a bounded device-side wait of a GEMM gave up");
    }
    return TUFRG_OK;
}

tufrg_status tufrg_mlp_train_step(tufrg_mlp *n, const float *d_X, const float *d_T, int batch, float lr, float *h_loss)
{
    if (!n || !(lr > 0)) return TUFRG_EINVAL;
    tufrg_status st = tufrg_mlp_gradients(n, d_X, d_T, batch, n->d_g, h_loss);
    if (st != TUFRG_OK) return st;
    n->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->adam_t), c2 = 1.f - std::pow(b2, (float)n->adam_t);
    adam_kernel<<<gsz(n->n_params), 256, 0, n->stream>>>(n->d_w, n->d_g, n->d_m, n->d_v, n->d_w16, n->n_params, lr, b1,
                                                           b2, 1e-8f, c1, c2);
    MK(cudaGetLastError(), "Adam");
    return TUFRG_OK;
}

}  // extern "C"

namespace tufrg {
void mlp_dims(const tufrg_mlp *n, int *n_in, int *n_out)
{
    *n_in = n->n_in;
    *n_out = n->n_out;
}

// Inference for the surrogate inside a model's right-hand side (stream-ordered, no sync); all kernels
// return at once while *skip != 0.
cudaError_t mlp_forward_on(tufrg_mlp *n, cudaStream_t s, const float *X, int batch, float *Y, const int *skip)
{
    cudaStream_t keep = n->stream;
    n->stream = s;
    const tufrg_status st = infer(n, X, batch, Y, skip);
    n->stream = keep;
    return st == TUFRG_OK ? cudaSuccess : cudaErrorUnknown;
}
}  // namespace tufrg

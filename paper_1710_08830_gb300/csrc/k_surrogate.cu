// Learned loop surrogate inside the right-hand side (an addition with no counterpart in the paper).
//
// For a split-precision two-band model with an attached network, every evaluation of the loops
//   1. builds 20 features per transfer momentum q: sin/cos(n q_x), sin/cos(n q_y) for n = 1..4 and the
//      standardised log T, alpha, t', mu of the model;
//   2. runs the network (BF16 weights, FP32 accumulation) for all q and un-standardises its output into
//      the compact loops, L = (y * std + mean) / T (the network learns T dF/dT, the flow variable);
//   3. evaluates the direct fine-mesh k-sum at n_check momenta and compares (relative Frobenius norm over
//      both channels); if the residual is at most the tolerance the surrogate loops are kept and the
//      direct k-sum over all q returns at once, otherwise the direct k-sum overwrites them.
// A failed check also switches the surrogate off until it is re-armed: at every entry point that
// evaluates loops and at the start of every flow.  Inside a flow (which runs from high to low T, where
// the loops sharpen and the network's error grows) the surrogate therefore serves an unbroken first
// stretch of the flow and the direct k-sum the rest, so the step controller sees at most one switch;
// once off, every surrogate kernel returns at once.  All decisions are taken on the device (flags read
// by the kernels), so the whole right-hand side stays capturable as a CUDA graph; accepted, rejected
// and skipped evaluations are counted on the device.
#include <cmath>
#include <cstring>
#include <exception>
#include <string>
#include <vector>

#include "tufrg_internal.cuh"

// the network object's layout is private to k_mlp.cu; only its sizes are needed here
extern "C" long long tufrg_mlp_num_params(const tufrg_mlp *net);
extern "C" tufrg_status tufrg_mlp_forward(tufrg_mlp *net, const float *d_X, int batch, float *d_Y);

namespace tufrg {
namespace {

constexpr int NFEAT = 20;

// feature standardisation of log T: (log T - centre) / scale, fixed for the flow range [0.02, 10]
constexpr double LOGT_C = -0.8, LOGT_S = 3.1;

__global__ void features_kernel(int Lq, const double *scal, double a, double tp, double mu, float *X, const int *off)
{
    if (*off) return;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Lq * Lq) return;
    const double qx = 2.0 * M_PI * (q / Lq) / Lq, qy = 2.0 * M_PI * (q % Lq) / Lq;
    float *x = X + (size_t)q * NFEAT;
    for (int n = 1; n <= 4; n++) {
        x[4 * (n - 1) + 0] = (float)sin(n * qx);
        x[4 * (n - 1) + 1] = (float)cos(n * qx);
        x[4 * (n - 1) + 2] = (float)sin(n * qy);
        x[4 * (n - 1) + 3] = (float)cos(n * qy);
    }
    x[16] = (float)((log(scal[0]) - LOGT_C) / LOGT_S);
    x[17] = (float)((a - 0.2) / 0.2);
    x[18] = (float)((tp + 0.15) / 0.15);
    x[19] = (float)((mu + 0.9) / 0.3);
}

// network output [q][((ch*nd + d)*16 + ab)*2 + re/im] -> compact loops of both channels
__global__ void unstandardise_kernel(const float *Y, const float *mean, const float *sd, const double *scal, int Nq,
                                     int nd, float2 *Lc32, double2 *Lc64, const int *off)
{
    if (*off) return;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // over 2 * Nq * nd * 16
    const size_t per = (size_t)nd * 16;
    if (i >= 2 * (size_t)Nq * per) return;
    const int ch = (int)(i / (Nq * per));
    const size_t r = i % (Nq * per);
    const int q = (int)(r / per);
    const size_t e = r % per;
    const size_t j = ((size_t)ch * per + e) * 2;
    const size_t no = 2 * per * 2;
    const double invT = 1.0 / scal[0];
    const double re = ((double)Y[(size_t)q * no + j] * sd[j] + mean[j]) * invT;
    const double im = ((double)Y[(size_t)q * no + j + 1] * sd[j + 1] + mean[j + 1]) * invT;
    Lc32[i] = make_float2((float)re, (float)im);
    Lc64[i] = make_double2(re, im);
}

// relative Frobenius residual of the surrogate at the check momenta; sets the accept flag flag[0] and,
// on failure, the off flag flag[1]
__global__ void check_kernel(const float2 *Lc32, const double2 *chk, const int *check_q, int n_check, int Nq, int nd,
                             double tol, int *flag, unsigned long long *count)
{
    if (flag[1]) {   // switched off earlier: direct k-sum
        if (threadIdx.x == 0) {
            flag[0] = 0;
            count[2] += 1;
        }
        return;
    }
    __shared__ double sn[256], sd[256];
    const size_t per = (size_t)nd * 16;
    double num = 0.0, den = 0.0;
    for (size_t i = threadIdx.x; i < 2 * (size_t)n_check * per; i += blockDim.x) {
        const int ch = (int)(i / (n_check * per));
        const size_t r = i % (n_check * per);
        const int c = (int)(r / per);
        const size_t e = r % per;
        const float2 s = Lc32[((size_t)ch * Nq + check_q[c]) * per + e];
        const double2 d = chk[i];
        const double dx = (double)s.x - d.x, dy = (double)s.y - d.y;
        num += dx * dx + dy * dy;
        den += d.x * d.x + d.y * d.y;
    }
    sn[threadIdx.x] = num;
    sd[threadIdx.x] = den;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sn[threadIdx.x] += sn[threadIdx.x + w];
            sd[threadIdx.x] += sd[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double res = sd[0] > 0.0 ? sqrt(sn[0] / sd[0]) : 0.0;
        const int ok = (res <= tol && isfinite(res)) ? 1 : 0;
        flag[0] = ok;
        flag[1] = ok ? 0 : 1;
        count[ok ? 0 : 1] += 1;
    }
}

}  // namespace

cudaError_t launch_loops_reduce_f32(tufrg_model *m, const float2 *part, int n_s, double2 *out64, float2 *out32,
                                    const int *skip);

cudaError_t launch_surrogate(tufrg_model *m, int channel_mask)
{
    (void)channel_mask;
    const int Nq = m->Nq, nd = m->nd;
    PhaseScope ps(m, PH_LOOPS, 0);
    const int *off = m->d_sur_flag + 1;
    features_kernel<<<(Nq + 127) / 128, 128, 0, m->stream>>>(m->Lq, m->d_scal, m->sur_params[0], m->sur_params[1],
                                                             m->sur_params[2], m->d_sur_X, off);
    TUFRG_CUDA_TRY(cudaGetLastError());
    TUFRG_CUDA_TRY(mlp_forward_on(m->sur, m->stream, m->d_sur_X, Nq, m->d_sur_Y, off));
    const size_t n = 2 * (size_t)Nq * nd * 16;
    unstandardise_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->d_sur_Y, m->d_sur_mean, m->d_sur_std,
                                                                            m->d_scal, Nq, nd, m->d_Lc32, m->d_Lc, off);
    TUFRG_CUDA_TRY(cudaGetLastError());
    // direct k-sum at the check momenta (both channels)
    const size_t cper = (size_t)m->n_check * nd * 16;
    for (int ch = 0; ch < 2; ch++) {
        TUFRG_CUDA_TRY(launch_loops2_ex(m, ch, m->d_check_q, m->n_check, m->d_chk_part, off));
        TUFRG_CUDA_TRY(launch_loops_reduce_f32(m, m->d_chk_part, m->n_check, m->d_chk + ch * cper, nullptr, off));
    }
    check_kernel<<<1, 256, 0, m->stream>>>(m->d_Lc32, m->d_chk, m->d_check_q, m->n_check, Nq, nd, m->sur_tol,
                                           m->d_sur_flag, m->d_sur_count);
    m->launches += 4;
    return cudaGetLastError();
}

cudaError_t surrogate_rearm(tufrg_model *m)
{
    if (!m->sur) return cudaSuccess;
    return cudaMemsetAsync(m->d_sur_flag + 1, 0, sizeof(int), m->stream);
}

}  // namespace tufrg

using namespace tufrg;

extern "C" {

tufrg_status tufrg_set_surrogate(tufrg_model *m, tufrg_mlp *net, const float *h_mean, const float *h_std,
                                 const double *h_feature_params, double resid_tol, int n_check, const int *h_check_q)
try {
    if (!m) return TUFRG_EINVAL;
    auto drop = [&]() {
        void *ptrs[] = {m->d_check_q, m->d_sur_X, m->d_sur_Y, m->d_sur_mean, m->d_sur_std, m->d_chk_part, m->d_chk,
                        m->d_sur_flag, m->d_sur_count};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        m->d_check_q = nullptr; m->d_sur_X = nullptr; m->d_sur_Y = nullptr; m->d_sur_mean = nullptr;
        m->d_sur_std = nullptr; m->d_chk_part = nullptr; m->d_chk = nullptr; m->d_sur_flag = nullptr;
        m->d_sur_count = nullptr;
        m->sur = nullptr;
    };
    cudaStreamSynchronize(m->stream);
    if (m->step_graph) {   // a captured flow step must be re-captured with (or without) the surrogate
        cudaGraphExecDestroy(m->step_graph);
        m->step_graph = nullptr;
    }
    drop();
    if (!net) return TUFRG_OK;
    if (!h_mean || !h_std || !h_feature_params || !h_check_q || n_check < 1 || n_check > m->Nq || !(resid_tol > 0)) {
        m->err = "tufrg_set_surrogate: bad arguments";
        return TUFRG_EINVAL;
    }
    if (m->regulator != TUFRG_REG_TEMPERATURE) {
        m->err = "the loop surrogate is trained on the temperature flow";
        return TUFRG_ENOTSUP;
    }
    if (!loops2_supported(m) || m->basis != TUFRG_BASIS_ORBITAL) {
        m->err = "the loop surrogate needs a split-precision two-band model in the orbital basis";
        return TUFRG_ENOTSUP;
    }
    const int n_out = 2 * m->nd * 16 * 2;
    for (int i = 0; i < n_check; i++)
        if (h_check_q[i] < 0 || h_check_q[i] >= m->Nq) {
            m->err = "tufrg_set_surrogate: check momentum out of range";
            return TUFRG_EINVAL;
        }
    cudaError_t failed = cudaSuccess;
    auto ck = [&](cudaError_t e, const char *w) {
        if (e != cudaSuccess) {
            m->err = std::string(w) + ": " + cudaGetErrorString(e);
            failed = e;
            (void)cudaGetLastError();
        }
        return e == cudaSuccess;
    };
    const size_t chk_part = (size_t)n_check * m->plan.n_partials * m->dxs.size() * 5 * 16;
    bool ok = ck(cudaMalloc(&m->d_check_q, sizeof(int) * n_check), "cudaMalloc") &&
              ck(cudaMalloc(&m->d_sur_X, sizeof(float) * m->Nq * NFEAT), "cudaMalloc") &&
              ck(cudaMalloc(&m->d_sur_Y, sizeof(float) * (size_t)m->Nq * n_out), "cudaMalloc") &&
              ck(cudaMalloc(&m->d_sur_mean, sizeof(float) * n_out), "cudaMalloc") &&
              ck(cudaMalloc(&m->d_sur_std, sizeof(float) * n_out), "cudaMalloc") &&
              ck(cudaMalloc(&m->d_chk_part, sizeof(float2) * chk_part), "cudaMalloc") &&
              ck(cudaMalloc(&m->d_chk, sizeof(double2) * 2 * (size_t)n_check * m->nd * 16), "cudaMalloc") &&
              ck(cudaMalloc(&m->d_sur_flag, 2 * sizeof(int)), "cudaMalloc") &&
              ck(cudaMalloc(&m->d_sur_count, 3 * sizeof(unsigned long long)), "cudaMalloc") &&
              ck(cudaMemcpy(m->d_check_q, h_check_q, sizeof(int) * n_check, cudaMemcpyHostToDevice), "copy") &&
              ck(cudaMemcpy(m->d_sur_mean, h_mean, sizeof(float) * n_out, cudaMemcpyHostToDevice), "copy") &&
              ck(cudaMemcpy(m->d_sur_std, h_std, sizeof(float) * n_out, cudaMemcpyHostToDevice), "copy") &&
              ck(cudaMemset(m->d_sur_flag, 0, 2 * sizeof(int)), "memset") &&
              ck(cudaMemset(m->d_sur_count, 0, 3 * sizeof(unsigned long long)), "memset");
    if (!ok) {
        drop();
        return failed == cudaErrorMemoryAllocation ? TUFRG_ENOMEM : TUFRG_ECUDA;
    }
    int nin = 0, nout = 0;
    mlp_dims(net, &nin, &nout);
    if (nin != NFEAT || nout != n_out) {
        drop();
        m->err = "surrogate network does not match the model (it must map 20 features to 2 x n_delta x 16 x 2)";
        return TUFRG_EINVAL;
    }
    m->sur = net;
    m->sur_tol = resid_tol;
    m->n_check = n_check;
    std::memcpy(m->sur_params, h_feature_params, sizeof(m->sur_params));
    // size the network's activation buffers for Nq rows now, so no allocation happens inside a capture
    if (tufrg_mlp_forward(net, m->d_sur_X, m->Nq, m->d_sur_Y) != TUFRG_OK) {
        drop();
        m->err = "surrogate network does not match the model (it must map 20 features to 2 x n_delta x 16 x 2)";
        return TUFRG_EINVAL;
    }
    cudaDeviceSynchronize();
    return TUFRG_OK;
} catch (const std::exception &ex) {
    // a host allocation that failed (the error message) becomes TUFRG_ENOMEM instead of crossing the C boundary
    if (m) {
        try {
            m->err = std::string("host allocation failed: ") + ex.what();
        } catch (...) {
            m->err.clear();
        }
    }
    return TUFRG_ENOMEM;
}

tufrg_status tufrg_surrogate_stats(tufrg_model *m, long long *accepted, long long *rejected, long long *skipped)
{
    if (!m) return TUFRG_EINVAL;
    unsigned long long c[3] = {0, 0, 0};
    if (m->d_sur_count) {
        if (cudaMemcpyAsync(c, m->d_sur_count, sizeof(c), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaStreamSynchronize(m->stream) != cudaSuccess) {
            (void)cudaGetLastError();
            return TUFRG_ECUDA;
        }
    }
    if (accepted) *accepted = (long long)c[0];
    if (rejected) *rejected = (long long)c[1];
    if (skipped) *skipped = (long long)c[2];
    return TUFRG_OK;
}

}  // extern "C"

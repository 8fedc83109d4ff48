// Dormand-Prince 5(4) stage combinations and the error norm on the device: FP64, or on the split path FP32 sums of the
// (exactly FP32) stage derivatives with the FP64 state update.
// The flow state is HBM resident; these kernels stream it once per stage.
#include <algorithm>

#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

struct StageArgs {
    const double *k[7];
    double a[7];
    int nk;
};

// out = y + h * sum_j a_j k_j  (element-wise over doubles), h read from the device flow state; the
// FP64 result goes to out and/or its FP32 rounding to out32 (either may be NULL)
__global__ void rk_combine_kernel(double *out, float *out32, const double *y, const FlowDev *fs, StageArgs s, size_t n)
{
    const double h = fs->h;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < s.nk; j++) acc = fma(s.a[j], s.k[j][i], acc);
        const double v = fma(h, acc, y[i]);
        if (out) out[i] = v;
        if (out32) out32[i] = narrow_f(v);
    }
}

// The same on the split path: the stage derivatives are exact FP32 values, so the weighted sum runs in FP32 (read back
// without rounding by narrow_f) and only the step y + h sum is FP64 (one fused operation per element: the state keeps
// its FP64 accumulation, the increment carries the FP32 accuracy of the derivatives)
__global__ void rk_combine_f32_kernel(double *out, float *out32, const double *y, const FlowDev *fs, StageArgs s, size_t n)
{
    const double h = fs->h;
    float a[7];
#pragma unroll
    for (int j = 0; j < 7; j++) a[j] = j < s.nk ? (float)s.a[j] : 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < 7; j++) {
            if (j >= s.nk) break;
            acc = fmaf(a[j], narrow_f(s.k[j][i]), acc);
        }
        const double v = fma(h, widen_f(acc), y[i]);
        if (out) out[i] = v;
        if (out32) out32[i] = narrow_f(v);
    }
}

__global__ void to_f32_kernel(const double2 *x, float2 *y, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        y[i] = make_float2(narrow_f(v.x), narrow_f(v.y));
    }
}

__global__ void round_f32_kernel(const double *x, float *y, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = narrow_f(x[i]);
}

// max over complex entries of |h sum_j e_j k_j| / (atol + rtol max(|y|, |yn|)); non-finite -> +inf
__global__ void rk_error_kernel(const double2 *y, const double2 *yn, const FlowDev *fs, StageArgs s, size_t n,
                                unsigned long long *out)
{
    const double h = fs->h, atol = fs->atol, rtol = fs->rtol;
    double mx = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double er = 0.0, ei = 0.0;
        for (int j = 0; j < s.nk; j++) {
            const double2 kv = reinterpret_cast<const double2 *>(s.k[j])[i];
            er = fma(s.a[j], kv.x, er);
            ei = fma(s.a[j], kv.y, ei);
        }
        const double ea = fabs(h) * sqrt(er * er + ei * ei);
        const double2 a = y[i], b = yn[i];
        const double ya = sqrt(a.x * a.x + a.y * a.y), yb = sqrt(b.x * b.x + b.y * b.y);
        double r = ea / (atol + rtol * fmax(ya, yb));
        if (!isfinite(r)) r = INFINITY;
        mx = fmax(mx, r);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// The same norm on the split path in FP32 arithmetic (this GPU's FP64 pipe, which the square roots and divisions
// above run on, is narrow): the stage derivatives there are FP32 results widened exactly, so their FP32 values are
// read back without rounding (narrow_f on the integer pipe); the weighted sums, magnitudes and the ratio are FP32,
// which is ample for a step-size control norm.  The maximum is published as the double of the FP32 value.
__global__ void rk_error_f32_kernel(const double2 *y, const double2 *yn, const FlowDev *fs, StageArgs s, size_t n,
                                    unsigned long long *out)
{
    const float h = fabsf((float)fs->h), atol = (float)fs->atol, rtol = (float)fs->rtol;
    float e[7];
#pragma unroll
    for (int j = 0; j < 7; j++) e[j] = j < s.nk ? (float)s.a[j] : 0.f;
    float mx = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float er = 0.f, ei = 0.f;
#pragma unroll
        for (int j = 0; j < 7; j++) {
            if (j >= s.nk) break;
            const double2 kv = reinterpret_cast<const double2 *>(s.k[j])[i];
            er = fmaf(e[j], narrow_f(kv.x), er);
            ei = fmaf(e[j], narrow_f(kv.y), ei);
        }
        const float ea = h * sqrtf(fmaf(er, er, ei * ei));
        const double2 a = y[i], b = yn[i];
        const float ax = narrow_f(a.x), ay = narrow_f(a.y), bx = narrow_f(b.x), by = narrow_f(b.y);
        const float ya = sqrtf(fmaf(ax, ax, ay * ay)), yb = sqrtf(fmaf(bx, bx, by * by));
        float r = ea / (atol + rtol * fmaxf(ya, yb));
        if (!isfinite(r)) r = INFINITY;
        mx = fmaxf(mx, r);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(out, (unsigned long long)__double_as_longlong((double)mx));
}

// temperature of stage j: T = exp(x + c_j h); the products are scaled by T (f = T dX/dT)
__global__ void stage_scalars_kernel(const FlowDev *fs, double cj, double *scal)
{
    const double T = exp(fs->x + cj * fs->h);
    scal[0] = T;
    scal[1] = T;
}

__global__ void flow_init_kernel(FlowDev *fs, const unsigned long long *red)
{
    const double amax = __longlong_as_double((long long)red[0]);
    fs->amax = amax;
    fs->amax_prev = amax;
    if (!isfinite(amax)) {
        fs->status = 4;
    } else if (amax > fs->stop) {   // already above the stop value at T0: critical before the first step
        fs->Tc = exp(fs->x);
        fs->status = 1;
    }
}

// Accept or reject the attempt just computed (error norm in red[2], max|A| at the candidate in red[0]).
__global__ void flow_decide_kernel(FlowDev *fs, const unsigned long long *red)
{
    fs->accepted = 0;
    if (fs->status != 0) return;
    const double err = __longlong_as_double((long long)red[2]);
    const double amax_new = __longlong_as_double((long long)red[0]);
    fs->tries++;
    fs->err = err;
    if (!isfinite(err) || !isfinite(amax_new)) {
        fs->status = 4;
        return;
    }
    if (err <= 1.0) {
        fs->x_prev = fs->x;
        fs->x += fs->h;
        fs->n_steps++;
        fs->amax = amax_new;
        fs->accepted = 1;
        double fac = err > 0.0 ? 0.9 * pow(err, -0.2) : 5.0;
        fac = fmin(5.0, fmax(0.2, fac));
        if (amax_new > fs->stop) {
            const double t = (fs->stop - fs->amax_prev) / (amax_new - fs->amax_prev);
            fs->Tc = exp(fs->x_prev + t * (fs->x - fs->x_prev));
            fs->status = 1;
            return;
        }
        fs->amax_prev = amax_new;
        if (fs->x <= fs->xend + 1e-14) {
            fs->status = 2;
            return;
        }
        fs->h *= fac;
    } else {
        fs->n_reject++;
        fs->h *= fmin(1.0, fmax(0.2, 0.9 * pow(err, -0.2)));
        if (fabs(fs->h) < 1e-12) {
            fs->status = 5;
            return;
        }
    }
    if (fs->x + fs->h < fs->xend) fs->h = fs->xend - fs->x;
    if (fs->tries >= fs->max_tries) fs->status = 3;
}

// FSAL commit of an accepted attempt: y <- y_n, k_1 <- k_7
__global__ void flow_commit_kernel(const FlowDev *fs, double2 *y, const double2 *yn, double2 *k0, const double2 *k6, size_t n)
{
    if (!fs->accepted) return;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        y[i] = yn[i];
        k0[i] = k6[i];
    }
}

int grid_for(const tufrg_model *m, size_t n)
{
    const size_t want = (n + 255) / 256;
    const size_t cap = (size_t)m->sm_count * 16;
    return (int)(want < cap ? want : cap);
}

}  // namespace

cudaError_t launch_rk_combine(tufrg_model *m, double2 *out, float2 *out32, const double2 *y, const FlowDev *fs,
                              const double *a, double2 *const *k, int nk, size_t n)
{
    StageArgs s{};
    s.nk = 0;
    for (int j = 0; j < nk; j++) {
        if (a[j] == 0.0) continue;
        s.k[s.nk] = reinterpret_cast<const double *>(k[j]);
        s.a[s.nk] = a[j];
        s.nk++;
    }
    const size_t nd = 2 * n;
    PhaseScope ps(m, PH_RK);
    if (m->precision == TUFRG_FP64)
        rk_combine_kernel<<<grid_for(m, nd), 256, 0, m->stream>>>(reinterpret_cast<double *>(out),
                                                                  reinterpret_cast<float *>(out32),
                                                                  reinterpret_cast<const double *>(y), fs, s, nd);
    else
        rk_combine_f32_kernel<<<grid_for(m, nd), 256, 0, m->stream>>>(reinterpret_cast<double *>(out),
                                                                      reinterpret_cast<float *>(out32),
                                                                      reinterpret_cast<const double *>(y), fs, s, nd);
    return cudaGetLastError();
}

__global__ void widen_f64_kernel(const float *in, double *out, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = widen_f(in[i]);
}

cudaError_t launch_widen_f64(const float *d_in, double *d_out, size_t n, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 8192);
    widen_f64_kernel<<<(unsigned)blocks, 256, 0, stream>>>(d_in, d_out, n);
    return cudaGetLastError();
}

cudaError_t launch_round_f32(const double *d_in, float *d_out, size_t n, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    const size_t blocks = std::min<size_t>((n + 255) / 256, 8192);
    round_f32_kernel<<<(unsigned)blocks, 256, 0, stream>>>(d_in, d_out, n);
    return cudaGetLastError();
}

// timed with the Fourier transform, the first reader of the copy
cudaError_t launch_to_f32(tufrg_model *m, const double2 *d_state, float2 *d_out, size_t n)
{
    PhaseScope ps(m, PH_DFT);
    to_f32_kernel<<<grid_for(m, n), 256, 0, m->stream>>>(d_state, d_out, n);
    return cudaGetLastError();
}

cudaError_t launch_rk_error(tufrg_model *m, const double2 *y, const double2 *yn, const FlowDev *fs, const double *e,
                            double2 *const *k, int nk, size_t n)
{
    StageArgs s{};
    s.nk = 0;
    for (int j = 0; j < nk; j++) {
        if (e[j] == 0.0) continue;
        s.k[s.nk] = reinterpret_cast<const double *>(k[j]);
        s.a[s.nk] = e[j];
        s.nk++;
    }
    TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_amax + 2, 0, sizeof(unsigned long long), m->stream));
    PhaseScope ps(m, PH_RK);
    if (m->precision == TUFRG_FP64)
        rk_error_kernel<<<grid_for(m, n), 256, 0, m->stream>>>(y, yn, fs, s, n, m->d_amax + 2);
    else
        rk_error_f32_kernel<<<grid_for(m, n), 256, 0, m->stream>>>(y, yn, fs, s, n, m->d_amax + 2);
    return cudaGetLastError();
}

cudaError_t launch_stage_scalars(tufrg_model *m, const FlowDev *fs, double cj)
{
    m->launches++;
    stage_scalars_kernel<<<1, 1, 0, m->stream>>>(fs, cj, m->d_scal);
    return cudaGetLastError();
}

cudaError_t launch_flow_init(tufrg_model *m, FlowDev *fs)
{
    m->launches++;
    flow_init_kernel<<<1, 1, 0, m->stream>>>(fs, m->d_amax);
    return cudaGetLastError();
}

cudaError_t launch_flow_decide(tufrg_model *m, FlowDev *fs)
{
    m->launches++;
    flow_decide_kernel<<<1, 1, 0, m->stream>>>(fs, m->d_amax);
    return cudaGetLastError();
}

cudaError_t launch_flow_commit(tufrg_model *m, const FlowDev *fs, double2 *y, const double2 *yn, double2 *k0,
                               const double2 *k6, size_t n)
{
    PhaseScope ps(m, PH_RK);
    flow_commit_kernel<<<grid_for(m, n), 256, 0, m->stream>>>(fs, y, yn, k0, k6, n);
    return cudaGetLastError();
}

}  // namespace tufrg

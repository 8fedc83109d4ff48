// Dormand-Prince 5(4) stage combinations and the error norm, FP64, on the device.
// The flow state is HBM resident; these kernels stream it once per stage.
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

struct StageArgs {
    const double *k[7];
    double a[7];
    int nk;
};

// out = y + h * sum_j a_j k_j  (element-wise over doubles)
__global__ void rk_combine_kernel(double *out, const double *y, double h, StageArgs s, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < s.nk; j++) acc = fma(s.a[j], s.k[j][i], acc);
        out[i] = fma(h, acc, y[i]);
    }
}

// max over complex entries of |h sum_j e_j k_j| / (atol + rtol max(|y|, |yn|)); non-finite -> +inf
__global__ void rk_error_kernel(const double2 *y, const double2 *yn, double h, StageArgs s, size_t n, double atol,
                                double rtol, unsigned long long *out)
{
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

int grid_for(const tufrg_model *m, size_t n)
{
    const size_t want = (n + 255) / 256;
    const size_t cap = (size_t)m->sm_count * 16;
    return (int)(want < cap ? want : cap);
}

}  // namespace

cudaError_t launch_rk_combine(tufrg_model *m, double2 *out, const double2 *y, double h, const double *a,
                              double2 *const *k, int nk, size_t n)
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
    rk_combine_kernel<<<grid_for(m, nd), 256, 0, m->stream>>>(reinterpret_cast<double *>(out),
                                                              reinterpret_cast<const double *>(y), h, s, nd);
    return cudaGetLastError();
}

cudaError_t launch_rk_error(tufrg_model *m, const double2 *y, const double2 *yn, double h, const double *e,
                            double2 *const *k, int nk, size_t n, double atol, double rtol)
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
    rk_error_kernel<<<grid_for(m, n), 256, 0, m->stream>>>(y, yn, h, s, n, atol, rtol, m->d_amax + 2);
    return cudaGetLastError();
}

}  // namespace tufrg

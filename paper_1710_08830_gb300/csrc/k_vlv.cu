// dX/dT(q) = c_X A_X(q) L_X(q) A_X(q): Sec. 4.2 Eq. RGE_spin (c_P = 1) and the orbital
// form of Eq. rge_Dmat (c_C = 2).  The M x M loop matrix is never stored: it is
// expanded from the compact loops, L[(R1,a),(R2,b)] = Lc[d(R1-R2)][a][b].
//
// Small M (<= 64, every N_s = 2 bond set): one CTA per (q, channel) holds A, L and
// the intermediate T = A L in shared memory and writes c * T A.  FP64 for the
// plain path; FP32 arithmetic on the FP32 copies for the split path.
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

template <typename C2> __device__ __forceinline__ void cfma(C2 &acc, C2 a, C2 b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

template <typename R>
__global__ void vlv_small_kernel(const typename cpx<R>::t *A, const typename cpx<R>::t *Lc, const int *dij, int Nq,
                                 int M, int nff, int ns2, int nd, int chmask, const double *scal, double2 *out)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sA = reinterpret_cast<C2 *>(smem_raw);
    C2 *sL = sA + M * M;
    C2 *sT = sL + M * M;
    const int q = blockIdx.x, ch = blockIdx.y;
    const size_t M2 = (size_t)M * M;
    double2 *o = out + ((size_t)ch * Nq + q) * M2;
    if (!((chmask >> ch) & 1)) {
        for (int i = threadIdx.x; i < (int)M2; i += blockDim.x) o[i] = make_double2(0.0, 0.0);
        return;
    }
    const C2 *a = A + ((size_t)ch * Nq + q) * M2;
    const C2 *lc = Lc + ((size_t)ch * Nq + q) * nd * ns2 * ns2;
    for (int i = threadIdx.x; i < (int)M2; i += blockDim.x) {
        sA[i] = a[i];
        const int r = i / M, c = i % M;
        const int d = dij[(r / ns2) * nff + c / ns2];
        sL[i] = lc[((size_t)d * ns2 + r % ns2) * ns2 + c % ns2];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (int)M2; i += blockDim.x) {
        const int r = i / M, c = i % M;
        C2 acc = mk(R(0), R(0));
        for (int k = 0; k < M; k++) cfma(acc, sA[r * M + k], sL[k * M + c]);
        sT[i] = acc;
    }
    __syncthreads();
    const double sc = (ch == 0 ? 1.0 : 2.0) * scal[1];   // c_P = 1, c_C = 2, times the output scale
    for (int i = threadIdx.x; i < (int)M2; i += blockDim.x) {
        const int r = i / M, c = i % M;
        C2 acc = mk(R(0), R(0));
        for (int k = 0; k < M; k++) cfma(acc, sT[r * M + k], sA[k * M + c]);
        o[i] = make_double2(sc * (double)acc.x, sc * (double)acc.y);
    }
}

}  // namespace

cudaError_t launch_vlv(tufrg_model *m, const double2 *d_A, int channel_mask, double2 *d_out)
{
    const int M = m->M;
    if (tc_supported(m)) return launch_vlv_tc(m, channel_mask, d_out);
    if (M > 64) return launch_vlv_large(m, d_A, channel_mask, d_out);
    const int ns2 = m->ns * m->ns;
    dim3 grid(m->Nq, 2);
    const int threads = 256;
    PhaseScope ps(m, PH_VLV);
    if (m->precision == TUFRG_FP64) {
        const size_t smem = 3 * sizeof(double2) * M * M;
        auto k = vlv_small_kernel<double>;
        if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, threads, smem, m->stream>>>(d_A, m->d_Lc, m->d_dij, m->Nq, M, m->nff, ns2, m->nd, channel_mask,
                                              m->d_scal, d_out);
    } else {
        const size_t smem = 3 * sizeof(float2) * M * M;
        auto k = vlv_small_kernel<float>;
        if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<grid, threads, smem, m->stream>>>(m->d_A32, m->d_Lc32, m->d_dij, m->Nq, M, m->nff, ns2, m->nd,
                                              channel_mask, m->d_scal, d_out);
    }
    return cudaGetLastError();
}

}  // namespace tufrg

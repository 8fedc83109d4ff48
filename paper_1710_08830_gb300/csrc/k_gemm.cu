// dX/dT(q) = c_X A_X(q) L_X(q) A_X(q) for large M (multi-orbital bond sets, M = N_ff N_s^2 > 64):
// Eq. RGE_spin (c_P = 1) and the orbital form of Eq. rge_Dmat (c_C = 2).
//
// Batched complex GEMM on CUDA cores, 64 x 64 output tiles, 16-deep K slices staged in shared
// memory, a 4 x 4 complex register tile per thread.  Pass 1 forms T = A L with the loop matrix
// gathered from the compact loops (L[(R1,a),(R2,b)] = Lc[d(R1-R2)][a][b], never stored); pass 2
// writes c * T A.  FP64 on the plain path, FP32 on the split path.
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

template <typename C2> __device__ __forceinline__ void cfma(C2 &acc, C2 a, C2 b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// C[q] = scale * A[q] * B[q]; B is either a plain matrix (Bm) or the loop matrix gathered from Lc.
template <typename R, bool GATHER, bool OUT64>
__global__ void __launch_bounds__(256) cgemm_kernel(const typename cpx<R>::t *A, const typename cpx<R>::t *Bm,
                                                    const typename cpx<R>::t *Lc, const int *dij, int M, int nff,
                                                    int ns2, int nd, double scale, const double *scal, const int *qlist,
                                                    void *Cout)
{
    using C2 = typename cpx<R>::t;
    __shared__ C2 As[BK][BM + 1];
    __shared__ C2 Bs[BK][BN + 1];
    const int q = qlist ? qlist[blockIdx.z] : blockIdx.z;
    const size_t M2 = (size_t)M * M;
    const C2 *a = A + (size_t)q * M2;
    const C2 *b = GATHER ? nullptr : Bm + (size_t)q * M2;
    const C2 *lc = GATHER ? Lc + (size_t)q * nd * ns2 * ns2 : nullptr;
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    if (scal) scale *= scal[1];
    C2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) acc[i][j] = mk(R(0), R(0));
    for (int k0 = 0; k0 < M; k0 += BK) {
        // A tile: rows row0..+BM, cols k0..+BK  (stored transposed, As[k][row])
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            const int r = e / BK, kk = e % BK;
            const int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < M && gk < M) ? a[(size_t)gr * M + gk] : mk(R(0), R(0));
        }
        // B tile: rows k0..+BK, cols col0..+BN
        for (int e = threadIdx.x; e < BK * BN; e += 256) {
            const int kk = e / BN, c = e % BN;
            const int gk = k0 + kk, gc = col0 + c;
            C2 v = mk(R(0), R(0));
            if (gk < M && gc < M) {
                if (GATHER) {
                    const int d = dij[(gk / ns2) * nff + gc / ns2];
                    v = lc[((size_t)d * ns2 + gk % ns2) * ns2 + gc % ns2];
                } else {
                    v = b[(size_t)gk * M + gc];
                }
            }
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            C2 av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; i++) av[i] = As[kk][ty * TM + i];
#pragma unroll
            for (int j = 0; j < TN; j++) bv[j] = Bs[kk][tx * TN + j];
#pragma unroll
            for (int i = 0; i < TM; i++)
#pragma unroll
                for (int j = 0; j < TN; j++) cfma(acc[i][j], av[i], bv[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
        for (int j = 0; j < TN; j++) {
            const int gr = row0 + ty * TM + i, gc = col0 + tx * TN + j;
            if (gr >= M || gc >= M) continue;
            const size_t o = (size_t)q * M2 + (size_t)gr * M + gc;
            if (OUT64)
                reinterpret_cast<double2 *>(Cout)[o] = make_double2(scale * (double)acc[i][j].x, scale * (double)acc[i][j].y);
            else
                reinterpret_cast<C2 *>(Cout)[o] = mk(R(scale * acc[i][j].x), R(scale * acc[i][j].y));
        }
}

template <typename R>
cudaError_t run(tufrg_model *m, const typename cpx<R>::t *A, const typename cpx<R>::t *Lc, int channel_mask,
                double2 *out, typename cpx<R>::t *Tbuf, const int *qlist, int nlist)
{
    const int M = m->M, ns2 = m->ns * m->ns;
    const size_t M2 = (size_t)M * M, lper = (size_t)m->Nq * m->nd * ns2 * ns2;
    const dim3 grid((M + BN - 1) / BN, (M + BM - 1) / BM, qlist ? nlist : m->Nq);
    for (int ch = 0; ch < 2; ch++) {
        double2 *o = out + (size_t)ch * m->Nq * M2;
        if (!((channel_mask >> ch) & 1)) {
            TUFRG_CUDA_TRY(cudaMemsetAsync(o, 0, sizeof(double2) * m->Nq * M2, m->stream));
            continue;
        }
        const auto *a = A + (size_t)ch * m->Nq * M2;
        cgemm_kernel<R, true, false><<<grid, 256, 0, m->stream>>>(a, nullptr, Lc + ch * lper, m->d_dij, M, m->nff,
                                                                  ns2, m->nd, 1.0, nullptr, qlist, Tbuf);
        TUFRG_CUDA_TRY(cudaGetLastError());
        cgemm_kernel<R, false, true><<<grid, 256, 0, m->stream>>>(Tbuf, a, nullptr, nullptr, M, m->nff, ns2, m->nd,
                                                                  ch == 0 ? 1.0 : 2.0, m->d_scal, qlist, o);
        TUFRG_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_vlv_large(tufrg_model *m, const double2 *d_A, int channel_mask, double2 *d_out, const int *qlist,
                             int nlist)
{
    PhaseScope ps(m, PH_VLV, 4);
    if (m->precision == TUFRG_FP64) return run<double>(m, d_A, m->d_Lc, channel_mask, d_out, m->d_T, qlist, nlist);
    return run<float>(m, m->d_A32, m->d_Lc32, channel_mask, d_out, reinterpret_cast<float2 *>(m->d_T), qlist, nlist);
}

}  // namespace tufrg

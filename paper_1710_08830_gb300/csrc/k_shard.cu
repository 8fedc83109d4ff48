// The right-hand side split over shards of transfer momenta (one shard per rank, Sec. 3.3).  Loops,
// projections and products of a momentum need only that momentum; the projections also need the lattice
// Fourier transform of the exchange propagators, X(R'') = (1/Nq) sum_u e^{i u.R''} X(u), a sum over the whole
// transfer mesh.  A shard forms its part of that sum over its own momenta (shard_dft_kernel); the parts are
// added across the shards (an all-reduce of 2 ncls M^2 complex numbers, done by the caller), and each shard
// then finishes its own momenta from the sum.
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

template <typename R> __device__ __forceinline__ typename cpx<R>::t ld_r(const double2 &v);
template <> __device__ __forceinline__ double2 ld_r<double>(const double2 &v) { return v; }
template <> __device__ __forceinline__ float2 ld_r<float>(const double2 &v) { return make_float2(narrow_f(v.x), narrow_f(v.y)); }

constexpr int SH_CPT = 8;   // classes per thread

// xr[ch][c][e] = inv_nq sum_i e^{i q_i.R''_c} X_local[ch][i][e] for the classes c0 .. c0 + SH_CPT of this CTA;
// grid (entries / 256, class chunks, 2 channels).  The split path rounds the state and the phases to FP32 and
// accumulates in FP32, like its full transform; the result is written in FP64.
template <typename R>
__global__ void shard_dft_kernel(const double2 *X, int n, const int *q_list, int M2, int ncls, const double2 *clsph,
                                 int chmask, double inv_nq, double2 *xr)
{
    using C2 = typename cpx<R>::t;
    const int e = blockIdx.x * blockDim.x + threadIdx.x, c0 = blockIdx.y * SH_CPT, ch = blockIdx.z;
    if (e >= M2) return;
    C2 acc[SH_CPT];
#pragma unroll
    for (int c = 0; c < SH_CPT; c++) acc[c] = mk(R(0), R(0));
    if ((chmask >> ch) & 1) {
        const double2 *src = X + (size_t)ch * n * M2 + e;
        for (int i = 0; i < n; i++) {
            const C2 x = ld_r<R>(src[(size_t)i * M2]);
            const double2 *ph = clsph + (size_t)q_list[i] * ncls + c0;
#pragma unroll
            for (int c = 0; c < SH_CPT; c++) {
                if (c0 + c >= ncls) break;
                const C2 p = ld_r<R>(ph[c]);
                acc[c].x = fma(p.x, x.x, fma(-p.y, x.y, acc[c].x));
                acc[c].y = fma(p.x, x.y, fma(p.y, x.x, acc[c].y));
            }
        }
    }
#pragma unroll
    for (int c = 0; c < SH_CPT; c++)
        if (c0 + c < ncls)
            xr[((size_t)ch * ncls + c0 + c) * M2 + e] = make_double2((double)acc[c].x * inv_nq, (double)acc[c].y * inv_nq);
}

// out_local[ch][i][e] = full[ch][q_i][e]
__global__ void shard_gather_kernel(const double2 *full, int Nq, int n, const int *q_list, size_t M2, double2 *out)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * (size_t)n * M2) return;
    const size_t e = t % M2;
    const int i = (int)((t / M2) % n), ch = (int)(t / (M2 * n));
    out[t] = full[((size_t)ch * Nq + q_list[i]) * M2 + e];
}

}  // namespace

cudaError_t launch_shard_dft(tufrg_model *m, const double2 *d_state_local, int n, const int *d_q, int mask, double2 *d_xr)
{
    const int M2 = m->M * m->M;
    const dim3 grid((M2 + 255) / 256, (m->ncls + SH_CPT - 1) / SH_CPT, 2);
    PhaseScope ps(m, PH_DFT);
    if (m->precision == TUFRG_FP64)
        shard_dft_kernel<double><<<grid, 256, 0, m->stream>>>(d_state_local, n, d_q, M2, m->ncls, m->d_clsph, mask,
                                                              1.0 / m->Nq, d_xr);
    else
        shard_dft_kernel<float><<<grid, 256, 0, m->stream>>>(d_state_local, n, d_q, M2, m->ncls, m->d_clsph, mask,
                                                             1.0 / m->Nq, d_xr);
    return cudaGetLastError();
}

cudaError_t launch_shard_gather(tufrg_model *m, const double2 *d_full, int n, const int *d_q, double2 *d_out)
{
    const size_t M2 = (size_t)m->M * m->M, total = 2 * (size_t)n * M2;
    m->launches++;
    shard_gather_kernel<<<(unsigned)((total + 255) / 256), 256, 0, m->stream>>>(d_full, m->Nq, n, d_q, M2, d_out);
    return cudaGetLastError();
}

cudaError_t launch_loops_list(tufrg_model *m, int mask, const int *d_list, int n)
{
    if (m->ns == 2 && m->precision == TUFRG_FP64) return launch_loops(m, mask, false);   // sums every momentum
    // the list takes the place of the orbit representatives: loops at the listed momenta only, in chunks of the
    // loop scratch's capacity
    const int cap = m->sym ? m->n_loop_q : m->Nq;
    const bool sym0 = m->sym;
    int *list0 = m->d_loop_list;
    const int n0 = m->n_loop_q;
    cudaError_t e = cudaSuccess;
    for (int c0 = 0; c0 < n && e == cudaSuccess; c0 += cap) {
        m->sym = true;
        m->d_loop_list = const_cast<int *>(d_list) + c0;
        m->n_loop_q = std::min(cap, n - c0);
        e = launch_loops(m, mask, true);
    }
    m->sym = sym0;
    m->d_loop_list = list0;
    m->n_loop_q = n0;
    return e;
}

}  // namespace tufrg

// Channel projections of Sec. 3.3 on the device.
//
//   X(R'') = (1/Nq) sum_u e^{i u.R''} X(u)                         (Fourier transform, after Eq. zw_1)
//   A_P = P^[V0] + P + P^[V^C] + P^[V^D]                            (Eq. sum_P)
//     P^[V^C]_{RR'}(s) =  sum_R'' e^{i s.R''} C^{R+R'',R'-R''}_{s1s2s3s4}(R'')        (Eq. proj_PD)
//     P^[V^D]_{RR'}(s) = -e^{i s.R'} sum_R'' e^{i s.R''} C^{R+R'',-R'-R''}_{s1s2s4s3}(R'')
//   A_C = C^[V0] + C^[V^P] + C + C^[V^D]
//     C^[V^P]_{RR'}(u) =  sum_R'' e^{i u.R''} P^{R+R'',R'-R''}_{s1s2s3s4}(R'')
//     C^[V^D]_{RR'}(u) = -sum_R'' e^{i u.R''} C^{R-R'+R'',R''}_{s1s2s4s3}(-R')        (Eq. proj_DC)
//
// The bond arithmetic of these sums is done once on the host into int32 gather
// tables (term lists per output bond pair (R, R')); the device kernel is a pure
// gather: one thread per output entry, each term one FP64 complex load from the
// Fourier-transformed source (L2 resident) times a phase from a [q][phase] table.
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int DFT_CPT = 8;   // bond classes per thread in the Fourier transform

__global__ void dft_kernel(const double2 *X, int Nq, size_t M2, int ncls, const double2 *clsph, double inv_nq,
                           double2 *Xr)
{
    const size_t ij = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c0 = blockIdx.y * DFT_CPT;
    const int ch = blockIdx.z;
    if (ij >= M2) return;
    const double2 *src = X + (size_t)ch * Nq * M2 + ij;
    double2 acc[DFT_CPT];
#pragma unroll
    for (int c = 0; c < DFT_CPT; c++) acc[c] = make_double2(0.0, 0.0);
    for (int u = 0; u < Nq; u++) {
        const double2 x = src[(size_t)u * M2];
        const double2 *ph = clsph + (size_t)u * ncls + c0;
#pragma unroll
        for (int c = 0; c < DFT_CPT; c++) {
            if (c0 + c < ncls) {
                const double2 p = __ldg(ph + c);
                acc[c].x = fma(p.x, x.x, fma(-p.y, x.y, acc[c].x));
                acc[c].y = fma(p.x, x.y, fma(p.y, x.x, acc[c].y));
            }
        }
    }
#pragma unroll
    for (int c = 0; c < DFT_CPT; c++)
        if (c0 + c < ncls)
            Xr[((size_t)ch * ncls + c0 + c) * M2 + ij] = make_double2(acc[c].x * inv_nq, acc[c].y * inv_nq);
}

__global__ void project_kernel(const double2 *X, const double2 *Xr, const double2 *V0, const int *gofs0,
                               const int *gofs1, const GatherTerm *gt0, const GatherTerm *gt1, const double2 *ph,
                               int nph, int Nq, int ns, int nff, int ncls, int chmask, double2 *A, float2 *A32,
                               unsigned long long *amax)
{
    const int ns2 = ns * ns, M = nff * ns2;
    const size_t M2 = (size_t)M * M;
    const size_t ij = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    const int ch = blockIdx.z;
    double mag = 0.0;
    if (ij < M2) {
        const int row = (int)(ij / M), col = (int)(ij % M);
        const int iR = row / ns2, rp = row % ns2, iRp = col / ns2, cp = col % ns2;
        // decode the orbital indices of this output entry
        int s1, s2, s3, s4;
        if (ch == 0) { s1 = rp / ns; s2 = rp % ns; s4 = cp / ns; s3 = cp % ns; }   // P: (s1,s2),(s4,s3)
        else         { s1 = rp / ns; s3 = rp % ns; s4 = cp / ns; s2 = cp % ns; }   // C: (s1,s3),(s4,s2)
        double2 val = make_double2(0.0, 0.0);
        if ((chmask >> ch) & 1) {
            val = X[((size_t)ch * Nq + q) * M2 + ij];
            if (iR == 0 && iRp == 0) {
                const double2 v0 = V0[((s1 * ns + s2) * ns + s3) * ns + s4];
                val.x += v0.x; val.y += v0.y;
            }
            const int *gofs = ch == 0 ? gofs0 : gofs1;
            const GatherTerm *gt = ch == 0 ? gt0 : gt1;
            const int b = gofs[iR * nff + iRp], e = gofs[iR * nff + iRp + 1];
            for (int t = b; t < e; t++) {
                const GatherTerm g = gt[t];
                int sch, sr, sc;
                double sgn;
                switch (g.kind) {
                case 0: sch = 1; sr = s1 * ns + s3; sc = s4 * ns + s2; sgn = 1.0; break;    // P <- C
                case 1: sch = 1; sr = s1 * ns + s4; sc = s3 * ns + s2; sgn = -1.0; break;   // P <- D
                case 2: sch = 0; sr = s1 * ns + s2; sc = s4 * ns + s3; sgn = 1.0; break;    // C <- P
                default: sch = 1; sr = s1 * ns + s4; sc = s3 * ns + s2; sgn = -1.0; break;  // C <- D
                }
                if (!((chmask >> sch) & 1)) continue;
                const double2 x = Xr[((size_t)sch * ncls + g.cls) * M2 + (size_t)(g.i1 * ns2 + sr) * M + g.i2 * ns2 + sc];
                const double2 p = ph[(size_t)q * nph + g.ph];
                val.x += sgn * (p.x * x.x - p.y * x.y);
                val.y += sgn * (p.x * x.y + p.y * x.x);
            }
        }
        A[((size_t)ch * Nq + q) * M2 + ij] = val;
        if (A32) A32[((size_t)ch * Nq + q) * M2 + ij] = make_float2((float)val.x, (float)val.y);
        mag = sqrt(val.x * val.x + val.y * val.y);
    }
    // max |A|: non-negative doubles order like their bit patterns
    for (int o = 16; o > 0; o >>= 1) mag = fmax(mag, __shfl_xor_sync(0xffffffffu, mag, o));
    if ((threadIdx.x & 31) == 0 && mag > 0.0) atomicMax(amax, (unsigned long long)__double_as_longlong(mag));
}

// Locate the maximum: every entry equal to the reduced maximum records its flat index (atomicMin keeps the first).
__global__ void amax_locate_kernel(const double2 *A, size_t n, const unsigned long long *amax, unsigned long long *where)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = A[i];
    const double mag = sqrt(v.x * v.x + v.y * v.y);
    if ((unsigned long long)__double_as_longlong(mag) == *amax) atomicMin(where, (unsigned long long)i);
}

}  // namespace

cudaError_t launch_dft(tufrg_model *m, const double2 *d_state, int channel_mask)
{
    const size_t M2 = (size_t)m->M * m->M;
    const int threads = 128;
    // both channels in one launch when both flow; otherwise only the one that does
    const int ch_lo = (channel_mask & 1) ? 0 : 1, ch_hi = (channel_mask & 2) ? 1 : 0;
    if (ch_lo > ch_hi) return cudaSuccess;
    dim3 grid((unsigned)((M2 + threads - 1) / threads), (m->ncls + DFT_CPT - 1) / DFT_CPT, ch_hi - ch_lo + 1);
    const size_t off = (size_t)ch_lo * m->Nq * M2;
    PhaseScope ps(m, PH_DFT);
    dft_kernel<<<grid, threads, 0, m->stream>>>(d_state + off, m->Nq, M2, m->ncls, m->d_clsph, 1.0 / m->Nq,
                                                 m->d_Xr + (size_t)ch_lo * m->ncls * M2);
    return cudaGetLastError();
}

cudaError_t launch_project(tufrg_model *m, const double2 *d_state, int channel_mask, double2 *d_A)
{
    const size_t M2 = (size_t)m->M * m->M;
    TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_amax, 0, sizeof(unsigned long long), m->stream));
    const int threads = 128;
    dim3 grid((unsigned)((M2 + threads - 1) / threads), m->Nq, 2);
    float2 *a32 = m->precision == TUFRG_FP64 ? nullptr : m->d_A32;
    PhaseScope ps(m, PH_PROJ);
    project_kernel<<<grid, threads, 0, m->stream>>>(d_state, m->d_Xr, m->d_V0, m->d_gofs[0], m->d_gofs[1],
                                                     m->d_gterms[0], m->d_gterms[1], m->d_ph, m->nph, m->Nq, m->ns,
                                                     m->nff, m->ncls, channel_mask, d_A, a32, m->d_amax);
    return cudaGetLastError();
}

cudaError_t launch_amax_locate(tufrg_model *m, const double2 *d_A, size_t n, double)
{
    TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_amax + 1, 0xff, sizeof(unsigned long long), m->stream));
    m->launches++;
    amax_locate_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(d_A, n, m->d_amax, m->d_amax + 1);
    return cudaGetLastError();
}

}  // namespace tufrg

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
// Fourier transform: one thread per matrix entry and a slice of the transfer mesh,
// a block of bond classes in registers, phases staged in shared memory; the
// slices are added in a fixed order by a second kernel (deterministic).  The
// state is read once from HBM; the split path accumulates in FP32.
//
// Projections: the bond arithmetic is done once on the host into int32 gather
// tables (terms per output bond pair (R, R')).  One CTA per (R, R', q-tile,
// channel) stages its term list in shared memory, so every warp walks the same
// list; threads cover the orbital pairs x transfer momenta of the tile.  Each
// term is one load from the (L2 resident) Fourier transform times a phase.
#include <algorithm>

#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

template <typename R> __device__ __forceinline__ typename cpx<R>::t ld_as(const double2 &v);
template <> __device__ __forceinline__ double2 ld_as<double>(const double2 &v) { return v; }
template <> __device__ __forceinline__ float2 ld_as<float>(const double2 &v) { return make_float2((float)v.x, (float)v.y); }

template <typename R, int CPT>
__global__ void dft_kernel(const double2 *X, int Nq, int M2, int ncls, int nchunk, const double2 *clsph, int u_per,
                           typename cpx<R>::t *part)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *ph = reinterpret_cast<C2 *>(smem_raw);   // [u_per][CPT]
    const int ch = blockIdx.z / nchunk, c0 = (blockIdx.z % nchunk) * CPT;
    const int u0 = blockIdx.y * u_per, u1 = min(Nq, u0 + u_per);
    for (int i = threadIdx.x; i < (u1 - u0) * CPT; i += blockDim.x) {
        const int u = u0 + i / CPT, c = c0 + i % CPT;
        ph[i] = c < ncls ? ld_as<R>(clsph[(size_t)u * ncls + c]) : mk(R(0), R(0));
    }
    __syncthreads();
    const int ij = blockIdx.x * blockDim.x + threadIdx.x;
    if (ij >= M2) return;
    C2 acc[CPT];
#pragma unroll
    for (int c = 0; c < CPT; c++) acc[c] = mk(R(0), R(0));
    const double2 *src = X + ((size_t)ch * Nq + u0) * M2 + ij;
    for (int u = u0; u < u1; u++, src += M2) {
        const C2 x = ld_as<R>(*src);
        const C2 *p = ph + (u - u0) * CPT;
#pragma unroll
        for (int c = 0; c < CPT; c++) {
            acc[c].x = fma(p[c].x, x.x, fma(-p[c].y, x.y, acc[c].x));
            acc[c].y = fma(p[c].x, x.y, fma(p[c].y, x.x, acc[c].y));
        }
    }
#pragma unroll
    for (int c = 0; c < CPT; c++)
        if (c0 + c < ncls) part[(((size_t)blockIdx.y * 2 + ch) * ncls + c0 + c) * M2 + ij] = acc[c];
}

template <typename R>
__global__ void dft_reduce_kernel(const typename cpx<R>::t *part, int nsplit, int ch_lo, int nch, int ncls, int M2,
                                  double inv_nq, typename cpx<R>::t *Xr)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // over nch * ncls * M2
    const size_t per = (size_t)ncls * M2;
    if (i >= (size_t)nch * per) return;
    const int ch = ch_lo + (int)(i / per);
    const size_t r = i % per;
    R sx = 0, sy = 0;
    for (int s = 0; s < nsplit; s++) {
        const auto v = part[((size_t)s * 2 + ch) * per + r];
        sx += v.x;
        sy += v.y;
    }
    Xr[(size_t)ch * per + r] = mk(R(sx * inv_nq), R(sy * inv_nq));
}

template <typename R>
__global__ void project_kernel(const double2 *X, const typename cpx<R>::t *Xr, const double2 *V0, const int *gofs0,
                               const int *gofs1, const GatherTerm *gt0, const GatherTerm *gt1,
                               const typename cpx<R>::t *ph, int nph, int Nq, int ns, int nff, int ncls, int chmask,
                               int qt, double2 *A, float2 *A32, unsigned long long *amax)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GatherTerm *terms = reinterpret_cast<GatherTerm *>(smem_raw);
    const int ns2 = ns * ns, ns4 = ns2 * ns2, M = nff * ns2;
    const size_t M2 = (size_t)M * M;
    const int pair = blockIdx.x, iR = pair / nff, iRp = pair % nff;
    const int q0 = blockIdx.y * qt;
    const int ch = blockIdx.z;
    const bool on = (chmask >> ch) & 1;
    const int *gofs = ch == 0 ? gofs0 : gofs1;
    const GatherTerm *gt = ch == 0 ? gt0 : gt1;
    const int tb = gofs[pair], nt = gofs[pair + 1] - tb;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) terms[t] = gt[tb + t];
    __syncthreads();
    double mag = 0.0;
    for (int item = threadIdx.x; item < ns4 * qt; item += blockDim.x) {
        const int q = q0 + item / ns4, combo = item % ns4;
        if (q >= Nq) continue;
        const int rp = combo / ns2, cp = combo % ns2;
        const int row = iR * ns2 + rp, col = iRp * ns2 + cp;
        int s1, s2, s3, s4;
        if (ch == 0) { s1 = rp / ns; s2 = rp % ns; s4 = cp / ns; s3 = cp % ns; }   // P: (s1,s2),(s4,s3)
        else         { s1 = rp / ns; s3 = rp % ns; s4 = cp / ns; s2 = cp % ns; }   // C: (s1,s3),(s4,s2)
        const size_t o = ((size_t)ch * Nq + q) * M2 + (size_t)row * M + col;
        double2 val = make_double2(0.0, 0.0);
        if (on) {
            val = X[o];
            if (iR == 0 && iRp == 0) {
                const double2 v0 = V0[((s1 * ns + s2) * ns + s3) * ns + s4];
                val.x += v0.x;
                val.y += v0.y;
            }
            R gx = 0, gy = 0;
            for (int t = 0; t < nt; t++) {
                const GatherTerm g = terms[t];
                int sch, sr, sc;
                R sgn;
                switch (g.kind) {
                case 0: sch = 1; sr = s1 * ns + s3; sc = s4 * ns + s2; sgn = R(1); break;    // P <- C
                case 1: sch = 1; sr = s1 * ns + s4; sc = s3 * ns + s2; sgn = R(-1); break;   // P <- D
                case 2: sch = 0; sr = s1 * ns + s2; sc = s4 * ns + s3; sgn = R(1); break;    // C <- P
                default: sch = 1; sr = s1 * ns + s4; sc = s3 * ns + s2; sgn = R(-1); break;  // C <- D
                }
                if (!((chmask >> sch) & 1)) continue;
                const C2 x = Xr[((size_t)sch * ncls + g.cls) * M2 + (size_t)(g.i1 * ns2 + sr) * M + g.i2 * ns2 + sc];
                const C2 p = ph[(size_t)q * nph + g.ph];
                gx += sgn * (p.x * x.x - p.y * x.y);
                gy += sgn * (p.x * x.y + p.y * x.x);
            }
            val.x += (double)gx;
            val.y += (double)gy;
        }
        A[o] = val;
        if (A32) A32[o] = make_float2((float)val.x, (float)val.y);
        mag = fmax(mag, sqrt(val.x * val.x + val.y * val.y));
    }
    // max |A|: non-negative doubles order like their bit patterns
    for (int off = 16; off > 0; off >>= 1) mag = fmax(mag, __shfl_xor_sync(0xffffffffu, mag, off));
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

template <typename R, int CPT>
cudaError_t dft_run(tufrg_model *m, const double2 *d_state, int ch_lo, int nch, typename cpx<R>::t *part,
                    typename cpx<R>::t *Xr)
{
    const int M2 = m->M * m->M;
    const int threads = 128;
    const int nchunk = (m->ncls + CPT - 1) / CPT;
    const int xb = (M2 + threads - 1) / threads;
    const int nsplit = m->dft_nsplit;
    const int u_per = (m->Nq + nsplit - 1) / nsplit;
    const size_t smem = sizeof(typename cpx<R>::t) * u_per * CPT;
    auto k = dft_kernel<R, CPT>;
    if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    {
        PhaseScope ps(m, PH_DFT, 2);
        dim3 grid(xb, nsplit, nch * nchunk);
        // channels are numbered from ch_lo inside the kernels
        k<<<grid, threads, smem, m->stream>>>(d_state + (size_t)ch_lo * m->Nq * M2, m->Nq, M2, m->ncls, nchunk,
                                               m->d_clsph, u_per, part);
        TUFRG_CUDA_TRY(cudaGetLastError());
        const size_t total = (size_t)nch * m->ncls * M2;
        dft_reduce_kernel<R><<<(unsigned)((total + 255) / 256), 256, 0, m->stream>>>(
            part, nsplit, 0, nch, m->ncls, M2, 1.0 / m->Nq, Xr + (size_t)ch_lo * m->ncls * M2);
    }
    return cudaGetLastError();
}

}  // namespace

int dft_plan_nsplit(const tufrg_model *m)
{
    const int xb = (m->M * m->M + 127) / 128;
    const int cpt = m->precision == TUFRG_FP64 ? 8 : 16;
    const int nchunk = (m->ncls + cpt - 1) / cpt;
    const long want = 4L * m->sm_count;
    long ns = (want + (long)xb * 2 * nchunk - 1) / ((long)xb * 2 * nchunk);
    if (ns < 1) ns = 1;
    if (ns > m->Nq) ns = m->Nq;
    return (int)ns;
}

cudaError_t launch_dft(tufrg_model *m, const double2 *d_state, int channel_mask)
{
    const int ch_lo = (channel_mask & 1) ? 0 : 1, ch_hi = (channel_mask & 2) ? 1 : 0;
    if (ch_lo > ch_hi) return cudaSuccess;
    const int nch = ch_hi - ch_lo + 1;
    if (m->precision == TUFRG_FP64)
        return dft_run<double, 8>(m, d_state, ch_lo, nch, reinterpret_cast<double2 *>(m->d_dftpart), m->d_Xr);
    return dft_run<float, 16>(m, d_state, ch_lo, nch, reinterpret_cast<float2 *>(m->d_dftpart), m->d_Xr32);
}

cudaError_t launch_project(tufrg_model *m, const double2 *d_state, int channel_mask, double2 *d_A)
{
    TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_amax, 0, sizeof(unsigned long long), m->stream));
    const int ns4 = m->ns * m->ns * m->ns * m->ns;
    const int qt = ns4 >= 128 ? 1 : 128 / ns4;
    dim3 grid(m->nff * m->nff, (m->Nq + qt - 1) / qt, 2);
    const size_t smem = sizeof(GatherTerm) * (size_t)std::max(1, m->max_terms);
    PhaseScope ps(m, PH_PROJ);
    if (m->precision == TUFRG_FP64) {
        project_kernel<double><<<grid, 128, smem, m->stream>>>(d_state, m->d_Xr, m->d_V0, m->d_gofs[0], m->d_gofs[1],
                                                               m->d_gterms[0], m->d_gterms[1], m->d_ph, m->nph, m->Nq,
                                                               m->ns, m->nff, m->ncls, channel_mask, qt, d_A, nullptr,
                                                               m->d_amax);
    } else {
        project_kernel<float><<<grid, 128, smem, m->stream>>>(d_state, m->d_Xr32, m->d_V0, m->d_gofs[0], m->d_gofs[1],
                                                              m->d_gterms[0], m->d_gterms[1], m->d_ph32, m->nph, m->Nq,
                                                              m->ns, m->nff, m->ncls, channel_mask, qt, d_A, m->d_A32,
                                                              m->d_amax);
    }
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

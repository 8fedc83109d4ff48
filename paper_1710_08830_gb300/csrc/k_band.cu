// Exchange propagators in the band basis (Sec. 3.4: Eqs. trafo_P, mat_trafo_P, mat_trafo_D), two-band models.
//
//   U^{RR'}_{s1 s2 n1 n2}(s) = (1/N) sum_k f_R(k) f*_R'(k) U_{s1 n1}(s - k) U_{s2 n2}(k)
//   X^{RR'}_{s1 s2 n1 n2}(u) = (1/N) sum_k f_R(k) f*_R'(k) U_{s1 n1}(k) U*_{s2 n2}(k - u)
//   P_band(s) = T_P^dagger P(s) T_P,  T_P[(R1,(a,b)),(R,(c,d))] = U^{R1 R}_{b a d c}(s)
//   C_band(u) = T_C^dagger C(u) T_C,  T_C[(R1,(a,b)),(R,(c,d))] = X^{R1 R}_{a b c d}(u)
//
// with f_R(k) = e^{-ik.R} and N = N_k (the fine mesh of the loops).  The transformation matrices depend on
// R1 - R only: band_trafo_kernel forms them compactly, Tc[ch][q][d][ij] (d the bond difference, ij the
// 16 orbital x band index combinations), with the loop kernels' separable phases: per fine-mesh column the
// sum over k_y with e^{-i k_y dy} for the distinct dy, then e^{-i k_x dx} per bond difference.
// band_apply_kernel expands them to M x M matrices in shared memory and forms T^dagger X T per momentum
// and channel.  Split models compute in FP32 from the FP32 eigenvectors, FP64 models in FP64.
#include <algorithm>

#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int BB_MAXDY = 16;    // distinct dy of the bond differences
constexpr int BB_MAXD = 128;    // bond differences
constexpr int BB_LANES = 8;     // fine-mesh columns handled side by side per index combination

template <typename R> __device__ __forceinline__ typename cpx<R>::t ldc(const double2 &v);
template <> __device__ __forceinline__ double2 ldc<double>(const double2 &v) { return v; }
template <> __device__ __forceinline__ float2 ldc<float>(const double2 &v) { return make_float2(narrow_f(v.x), narrow_f(v.y)); }
__device__ __forceinline__ double2 wide2(double2 v) { return v; }
__device__ __forceinline__ double2 wide2(float2 v) { return make_double2(widen_f(v.x), widen_f(v.y)); }

struct BandTabs {
    int ndy, dy[BB_MAXDY];          // distinct dy values, reduced modulo Lf into [0, Lf)
    int nd, dx[BB_MAXD];            // bond differences sorted by their dy: dx, and
    int orig[BB_MAXD];              //   the index in the model's difference list
    int ofs[BB_MAXDY + 1];          //   the group of dy[i] is [ofs[i], ofs[i+1])
};

// Grid (q, channel); 128 threads = 16 index combinations ij = ((a 2 + b) 2 + c) 2 + d x 8 column lanes.
template <typename R>
__global__ void __launch_bounds__(16 * BB_LANES) band_trafo_kernel(const typename cpx<R>::t *__restrict__ U, int Lq,
                                                                 int nc, int Lf, BandTabs tb,
                                                                 typename cpx<R>::t *__restrict__ Tc)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *ptab = reinterpret_cast<C2 *>(smem_raw);       // [Lf] e^{-2 pi i n / Lf}
    C2 *acc = ptab + Lf;                                // [nd][128] per-thread sums over its columns
    const int q = blockIdx.x, ch = blockIdx.y, Nq = gridDim.x;
    for (int n = threadIdx.x; n < Lf; n += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)n / (double)Lf, &sn, &cs);
        ptab[n] = mk(R(cs), R(-sn));
    }
    for (int i = threadIdx.x; i < tb.nd * (int)blockDim.x; i += blockDim.x) acc[i] = mk(R(0), R(0));
    __syncthreads();
    const int ij = threadIdx.x / BB_LANES, lane = threadIdx.x % BB_LANES;
    const int a = (ij >> 3) & 1, b = (ij >> 2) & 1, c = (ij >> 1) & 1, d = ij & 1;
    const int sx = (q / Lq) * nc, sy = (q % Lq) * nc;
    for (int kx = lane; kx < Lf; kx += BB_LANES) {
        // the other momentum's column: s - k (P) or k - u (C)
        const int ox = ch == 0 ? (sx - kx + Lf) % Lf : (kx - sx + Lf) % Lf;
        C2 z[BB_MAXDY];
        int pn[BB_MAXDY];
#pragma unroll
        for (int i = 0; i < BB_MAXDY; i++) { z[i] = mk(R(0), R(0)); pn[i] = 0; }
        for (int ky = 0; ky < Lf; ky++) {
            int oy = ch == 0 ? sy - ky : ky - sy;
            if (oy < 0) oy += Lf;
            const C2 u1 = U[((size_t)kx * Lf + ky) * 4 + a * 2 + c];     // U_{a c}(k)
            const C2 u2 = U[((size_t)ox * Lf + oy) * 4 + b * 2 + d];     // U_{b d}(other)
            // P: U_{b d}(s - k) U_{a c}(k); C: U_{a c}(k) conj(U_{b d}(k - u))
            const C2 v = ch == 0 ? mk(u1.x * u2.x - u1.y * u2.y, u1.x * u2.y + u1.y * u2.x)
                                 : mk(u1.x * u2.x + u1.y * u2.y, u1.y * u2.x - u1.x * u2.y);
#pragma unroll
            for (int i = 0; i < BB_MAXDY; i++) {
                if (i >= tb.ndy) break;
                const C2 p = ptab[pn[i]];
                z[i].x = fma(p.x, v.x, fma(-p.y, v.y, z[i].x));
                z[i].y = fma(p.x, v.y, fma(p.y, v.x, z[i].y));
                pn[i] += tb.dy[i];   // (ky dy) mod Lf, advanced by one row
                if (pn[i] >= Lf) pn[i] -= Lf;
            }
        }
        // e^{-i k_x dx} z(dy) into this thread's sums, bond differences grouped by their dy
#pragma unroll
        for (int i = 0; i < BB_MAXDY; i++) {
            if (i >= tb.ndy) break;
            for (int e = tb.ofs[i]; e < tb.ofs[i + 1]; e++) {
                const C2 p = ptab[(((long)kx * tb.dx[e]) % Lf + Lf) % Lf];
                C2 &o = acc[e * blockDim.x + threadIdx.x];
                o.x = fma(p.x, z[i].x, fma(-p.y, z[i].y, o.x));
                o.y = fma(p.x, z[i].y, fma(p.y, z[i].x, o.y));
            }
        }
    }
    __syncthreads();
    const R inv_nk = R(1.0 / ((double)Lf * Lf));
    for (int o = threadIdx.x; o < tb.nd * 16; o += blockDim.x) {
        const int e = o / 16, c16 = o % 16;
        R re = 0, im = 0;
        for (int l = 0; l < BB_LANES; l++) {
            const C2 v = acc[e * blockDim.x + c16 * BB_LANES + l];
            re += v.x;
            im += v.y;
        }
        Tc[(((size_t)ch * Nq + q) * tb.nd + tb.orig[e]) * 16 + c16] = mk(re * inv_nk, im * inv_nk);
    }
}

// Grid (q, channel): T^dagger X T with T expanded from Tc (T[(R1,(a,b)),(R,(c,d))] = Tc[d(R1 - R)][abcd]).
template <typename R>
__global__ void __launch_bounds__(256) band_apply_kernel(const double2 *__restrict__ X, const typename cpx<R>::t *__restrict__ Tc,
                                                         const int *__restrict__ dij, int nff, int nd, double2 *__restrict__ out)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = 4 * nff, M2 = M * M, q = blockIdx.x, ch = blockIdx.y, Nq = gridDim.x;
    C2 *sX = reinterpret_cast<C2 *>(smem_raw), *sT = sX + M2, *sW = sT + M2;
    const double2 *x = X + ((size_t)ch * Nq + q) * M2;
    const C2 *tc = Tc + ((size_t)ch * Nq + q) * nd * 16;
    for (int i = threadIdx.x; i < M2; i += blockDim.x) {
        const int r = i / M, c = i % M;
        sX[i] = ldc<R>(x[i]);
        const int ab = r & 3, cd = c & 3;   // pair indices (a, b) and (c, d)
        sT[i] = tc[dij[(r >> 2) * nff + (c >> 2)] * 16 + ab * 4 + cd];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M2; i += blockDim.x) {   // W = X T
        const int r = i / M, c = i % M;
        C2 acc = mk(R(0), R(0));
        for (int j = 0; j < M; j++) {
            const C2 u = sX[r * M + j], v = sT[j * M + c];
            acc.x = fma(u.x, v.x, fma(-u.y, v.y, acc.x));
            acc.y = fma(u.x, v.y, fma(u.y, v.x, acc.y));
        }
        sW[i] = acc;
    }
    __syncthreads();
    double2 *o = out + ((size_t)ch * Nq + q) * M2;
    for (int i = threadIdx.x; i < M2; i += blockDim.x) {   // out = T^dagger W
        const int r = i / M, c = i % M;
        C2 acc = mk(R(0), R(0));
        for (int j = 0; j < M; j++) {
            const C2 u = sT[j * M + r], v = sW[j * M + c];   // conj(T[j][r]) W[j][c]
            acc.x = fma(u.x, v.x, fma(u.y, v.y, acc.x));
            acc.y = fma(u.x, v.y, fma(-u.y, v.x, acc.y));
        }
        o[i] = wide2(acc);
    }
}

template <typename R>
cudaError_t band_run(tufrg_model *m, const typename cpx<R>::t *U, const BandTabs &tb, const double2 *d_state, double2 *d_out)
{
    using C2 = typename cpx<R>::t;
    C2 *Tc = reinterpret_cast<C2 *>(m->d_band_tc);
    const size_t s1 = sizeof(C2) * (m->Lf + (size_t)tb.nd * 16 * BB_LANES);
    auto k1 = band_trafo_kernel<R>;
    if (s1 > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1));
    k1<<<dim3(m->Nq, 2), 16 * BB_LANES, s1, m->stream>>>(U, m->Lq, m->nc, m->Lf, tb, Tc);
    TUFRG_CUDA_TRY(cudaGetLastError());
    const size_t s2 = 3 * sizeof(C2) * (size_t)m->M * m->M;
    auto k2 = band_apply_kernel<R>;
    if (s2 > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2));
    k2<<<dim3(m->Nq, 2), 256, s2, m->stream>>>(d_state, Tc, m->d_dij, m->nff, m->nd, d_out);
    m->launches += 2;
    return cudaGetLastError();
}

}  // namespace

namespace {
// S[ch][q][e] = v0d[ch][e] for every q: the bare vertex's projections in the orbital basis (onsite)
__global__ void bare_state_kernel(const double2 *v0d0, const double2 *v0d1, int Nq, size_t M2, double2 *S)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * (size_t)Nq * M2) return;
    const size_t e = t % M2;
    S[t] = (t / M2) < (size_t)Nq ? v0d0[e] : v0d1[e];
}

template <typename C2>
__global__ void unit_eigvec_kernel(C2 *U, size_t Nk, int ns)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Nk * ns * ns) return;
    const int tl = (int)(t % ((size_t)ns * ns));
    U[t] = mk((decltype(U[t].x))(tl / ns == tl % ns ? 1 : 0), (decltype(U[t].x))0);
}
}  // namespace

cudaError_t setup_band_flow(tufrg_model *m)
{
    const size_t M2 = (size_t)m->M * m->M, n = 2 * (size_t)m->Nq * M2;
    double2 *S = nullptr;
    TUFRG_CUDA_TRY(cudaMalloc(&S, sizeof(double2) * n));
    cudaError_t e = cudaMalloc(&m->d_v0q, sizeof(double2) * n);
    if (e == cudaSuccess) {
        bare_state_kernel<<<(unsigned)((n + 255) / 256), 256, 0, m->stream>>>(m->d_v0d[0], m->d_v0d[1], m->Nq, M2, S);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_band_basis(m, S, m->d_v0q);   // with the model's eigenvectors
    if (e == cudaSuccess && m->precision != TUFRG_FP64) {
        e = cudaMalloc(&m->d_v0q32, sizeof(float2) * n);
        if (e == cudaSuccess) e = launch_to_f32(m, m->d_v0q, m->d_v0q32, n);
    }
    // the loops of the band basis: unit eigenvectors (stream ordered after the transformation above)
    const size_t nu = (size_t)m->Nk * m->ns * m->ns;
    if (e == cudaSuccess) {
        unit_eigvec_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, m->stream>>>(m->d_U, (size_t)m->Nk, m->ns);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && m->d_U32) {
        unit_eigvec_kernel<<<(unsigned)((nu + 255) / 256), 256, 0, m->stream>>>(m->d_U32, (size_t)m->Nk, m->ns);
        e = cudaGetLastError();
    }
    cudaStreamSynchronize(m->stream);
    cudaFree(S);
    return e;
}

bool band_basis_supported(const tufrg_model *m)
{
    const size_t c2 = m->precision == TUFRG_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t s1 = c2 * (m->Lf + (size_t)m->nd * 16 * BB_LANES), s2 = 3 * c2 * (size_t)m->M * m->M;
    return m->ns == 2 && m->M <= 64 && m->nd <= BB_MAXD && (int)m->dys.size() <= BB_MAXDY && s1 <= 227 * 1024 &&
           s2 <= 227 * 1024;
}

cudaError_t launch_band_basis(tufrg_model *m, const double2 *d_state, double2 *d_out)
{
    BandTabs tb{};
    tb.ndy = (int)m->dys.size();
    tb.nd = m->nd;
    int pos = 0;
    for (int i = 0; i < tb.ndy; i++) {
        tb.dy[i] = ((m->dys[i] % m->Lf) + m->Lf) % m->Lf;
        tb.ofs[i] = pos;
        for (int e = 0; e < m->nd; e++)
            if (m->deltas[2 * e + 1] == m->dys[i]) {
                tb.dx[pos] = m->deltas[2 * e];
                tb.orig[pos] = e;
                pos++;
            }
    }
    tb.ofs[tb.ndy] = pos;
    const bool fp64 = m->precision == TUFRG_FP64;
    if (!m->d_band_tc)
        TUFRG_CUDA_TRY(cudaMalloc(&m->d_band_tc, (fp64 ? sizeof(double2) : sizeof(float2)) * 2 * (size_t)m->Nq * m->nd * 16));
    if (fp64) return band_run<double>(m, m->d_U, tb, d_state, d_out);
    return band_run<float>(m, m->d_U32, tb, d_state, d_out);
}

}  // namespace tufrg

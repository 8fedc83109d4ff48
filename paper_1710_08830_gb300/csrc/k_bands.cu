// Band structure on the fine mesh (FP64) and the per-temperature Fermi tables.
//
// H(k) = sum_R t_R e^{i k.R} is diagonalised once per model (the temperature
// flow leaves it unchanged): H U = U diag(E), E ascending (Sec. 3.1, Eq. trafo
// uses the columns of U).  N_s = 2 uses the closed form of a Hermitian 2x2;
// other N_s use a cyclic complex Jacobi iteration in registers/local memory,
// one thread per k-point.  The Fermi tables hold, per (k, band) and per
// temperature, e = E - mu, g = df/dT and gp = dg/de (Eqs. disc_2a, disc_2b
// differentiated in T); every transcendental of the loop sums lives here.
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

__device__ __forceinline__ double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cj(double2 a) { return make_double2(a.x, -a.y); }

// H(k) from the hopping list; the phase exponent is reduced mod Lf first so
// that lattice-equivalent phases are computed from the same argument.
template <int NS>
__device__ void bloch_h(const int *hopR, const double2 *hopt, int nhop, int Lf, int kx, int ky, double2 *H)
{
    for (int i = 0; i < NS * NS; i++) H[i] = make_double2(0.0, 0.0);
    for (int h = 0; h < nhop; h++) {
        long n = ((long)kx * hopR[2 * h] + (long)ky * hopR[2 * h + 1]) % Lf;
        if (n < 0) n += Lf;
        double sn, cs;
        sincospi(2.0 * (double)n / (double)Lf, &sn, &cs);
        const double2 ph = make_double2(cs, sn);
        for (int i = 0; i < NS * NS; i++) {
            double2 p = cm(hopt[(size_t)h * NS * NS + i], ph);
            H[i].x += p.x;
            H[i].y += p.y;
        }
    }
}

// Closed-form eigensystem of [[a, b], [conj(b), d]].
__device__ void eig2(const double2 *H, double *E, double2 *U)
{
    const double a = H[0].x, d = H[3].x;
    const double2 b = H[1];
    const double m = 0.5 * (a + d), del = 0.5 * (a - d);
    const double bb = b.x * b.x + b.y * b.y;
    const double r = sqrt(del * del + bb);
    E[0] = m - r;
    E[1] = m + r;
    if (r == 0.0) {   // exactly degenerate and diagonal: keep the orbital basis
        U[0] = make_double2(1, 0); U[1] = make_double2(0, 0);
        U[2] = make_double2(0, 0); U[3] = make_double2(1, 0);
        return;
    }
    if (del >= 0.0) {
        // upper: (del + r, conj b), lower: (-b, del + r)
        const double p = del + r, n = 1.0 / sqrt(p * p + bb);
        U[0] = make_double2(-b.x * n, -b.y * n);   // row 0, lower band
        U[1] = make_double2(p * n, 0.0);           // row 0, upper band
        U[2] = make_double2(p * n, 0.0);           // row 1, lower band
        U[3] = make_double2(b.x * n, -b.y * n);    // row 1, upper band
    } else {
        // lower: (del - r, conj b), upper: (b, r - del)
        const double p = r - del, n = 1.0 / sqrt(p * p + bb);
        U[0] = make_double2(-p * n, 0.0);
        U[1] = make_double2(b.x * n, b.y * n);
        U[2] = make_double2(b.x * n, -b.y * n);
        U[3] = make_double2(p * n, 0.0);
    }
}

// Cyclic complex Jacobi: A <- V^H A V until the off-diagonal part is negligible.
template <int NS>
__device__ void eig_jacobi(double2 *A, double *E, double2 *V)
{
    for (int i = 0; i < NS; i++)
        for (int j = 0; j < NS; j++) V[i * NS + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    double nrm = 0.0;
    for (int i = 0; i < NS * NS; i++) nrm += A[i].x * A[i].x + A[i].y * A[i].y;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0;
        for (int p = 0; p < NS; p++)
            for (int q = p + 1; q < NS; q++) off += A[p * NS + q].x * A[p * NS + q].x + A[p * NS + q].y * A[p * NS + q].y;
        if (off <= 1e-30 * nrm) break;
        for (int p = 0; p < NS - 1; p++)
            for (int q = p + 1; q < NS; q++) {
                const double2 apq = A[p * NS + q];
                const double r = sqrt(apq.x * apq.x + apq.y * apq.y);
                if (r < 1e-300) continue;
                // rotation G in the (p,q) plane with G^H A G zeroing A_pq:
                //   G_pp = c, G_pq = s e, G_qp = -s conj(e), G_qq = c,  e = apq / |apq|
                const double2 e = make_double2(apq.x / r, apq.y / r);
                const double th = (A[q * NS + q].x - A[p * NS + p].x) / (2.0 * r);
                const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                const double2 se = make_double2(s * e.x, s * e.y);
                // columns: A <- A G
                for (int k = 0; k < NS; k++) {
                    const double2 akp = A[k * NS + p], akq = A[k * NS + q];
                    const double2 t1 = cm(akq, cj(se));
                    const double2 t2 = cm(akp, se);
                    A[k * NS + p] = make_double2(c * akp.x - t1.x, c * akp.y - t1.y);
                    A[k * NS + q] = make_double2(t2.x + c * akq.x, t2.y + c * akq.y);
                    const double2 vkp = V[k * NS + p], vkq = V[k * NS + q];
                    const double2 u1 = cm(vkq, cj(se));
                    const double2 u2 = cm(vkp, se);
                    V[k * NS + p] = make_double2(c * vkp.x - u1.x, c * vkp.y - u1.y);
                    V[k * NS + q] = make_double2(u2.x + c * vkq.x, u2.y + c * vkq.y);
                }
                // rows: A <- G^H A
                for (int k = 0; k < NS; k++) {
                    const double2 apk = A[p * NS + k], aqk = A[q * NS + k];
                    const double2 t1 = cm(se, aqk);
                    const double2 t2 = cm(cj(se), apk);
                    A[p * NS + k] = make_double2(c * apk.x - t1.x, c * apk.y - t1.y);
                    A[q * NS + k] = make_double2(t2.x + c * aqk.x, t2.y + c * aqk.y);
                }
                A[p * NS + q] = make_double2(0, 0);
                A[q * NS + p] = make_double2(0, 0);
            }
    }
    for (int i = 0; i < NS; i++) E[i] = A[i * NS + i].x;
    for (int i = 0; i < NS; i++) {   // ascending order
        int mn = i;
        for (int j = i + 1; j < NS; j++) if (E[j] < E[mn]) mn = j;
        if (mn != i) {
            const double te = E[i]; E[i] = E[mn]; E[mn] = te;
            for (int k = 0; k < NS; k++) { const double2 tv = V[k * NS + i]; V[k * NS + i] = V[k * NS + mn]; V[k * NS + mn] = tv; }
        }
    }
}

template <int NS>
__global__ void bands_kernel(const int *hopR, const double2 *hopt, int nhop, int Lf, double *E, double2 *U, float2 *U32)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Lf * Lf) return;
    double2 H[NS * NS], V[NS * NS];
    double ev[NS];
    bloch_h<NS>(hopR, hopt, nhop, Lf, k / Lf, k % Lf, H);
    if (NS == 2) eig2(H, ev, V);
    else eig_jacobi<NS>(H, ev, V);
    for (int l = 0; l < NS; l++) E[(size_t)k * NS + l] = ev[l];
    for (int i = 0; i < NS * NS; i++) {
        U[(size_t)k * NS * NS + i] = V[i];
        if (U32) U32[(size_t)k * NS * NS + i] = make_float2((float)V[i].x, (float)V[i].y);
    }
}

// f = 1/(e^{e/T}+1), g = df/dT = (e/T^2) f(1-f), gp = dg/de, all with z = e^{-|e|/T} (no overflow).
__device__ __forceinline__ void fermi_g(double e, double T, double &f, double &g, double &gp)
{
    const double x = e / T, ax = fabs(x);
    const double z = exp(-ax);
    const double h = z / ((1.0 + z) * (1.0 + z));
    f = e > 0 ? z / (1.0 + z) : 1.0 / (1.0 + z);
    g = x / T * h;
    gp = h / (T * T) * (1.0 - ax * (1.0 - z) / (1.0 + z));
}

__global__ void fermi_kernel(const double *E, int n, double mu, const double *scal, FermiEntry *ft, FermiEntry32 *ft32)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double T = scal[0];
    const double e = E[i] - mu;
    double f, g, gp;
    fermi_g(e, T, f, g, gp);
    ft[i] = FermiEntry{e, g, gp};
    if (ft32) ft32[i] = FermiEntry32{(float)e, (float)g, (float)gp, 0.f};
}

// Momentum-shell tables: (e, f, h) with h = f (1 - f) / T at the fixed temperature T (once per model).
__global__ void fermi_shell_kernel(const double *E, int n, double mu, double T, FermiEntry *ft, FermiEntry32 *ft32)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double e = E[i] - mu, z = exp(-fabs(e) / T);
    const double f = e > 0 ? z / (1.0 + z) : 1.0 / (1.0 + z), h = z / ((1.0 + z) * (1.0 + z)) / T;
    ft[i] = FermiEntry{e, f, h};
    if (ft32) ft32[i] = FermiEntry32{(float)e, (float)f, (float)h, 0.f};
}

// n(mu) partial sums: fixed-order tree in each block, then one block sums the partials.
__global__ void density_partial(const double *E, int n, double mu, double T, double *part)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double f, g, gp;
        fermi_g(E[i] - mu, T, f, g, gp);
        s += f;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void density_final(double *part, int nb)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nb; i++) s += part[i];
        part[nb] = s;
    }
}

}  // namespace

cudaError_t launch_bands(tufrg_model *m)
{
    const int n = m->Nk;
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    float2 *u32 = m->precision == TUFRG_FP64 ? nullptr : m->d_U32;
    m->launches++;
    switch (m->ns) {
    case 2: bands_kernel<2><<<blocks, threads, 0, m->stream>>>(m->d_hopR, m->d_hopt, m->nhop, m->Lf, m->d_E, m->d_U, u32); break;
    case 4: bands_kernel<4><<<blocks, threads, 0, m->stream>>>(m->d_hopR, m->d_hopt, m->nhop, m->Lf, m->d_E, m->d_U, u32); break;
    case 6: bands_kernel<6><<<blocks, threads, 0, m->stream>>>(m->d_hopR, m->d_hopt, m->nhop, m->Lf, m->d_E, m->d_U, u32); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

__global__ void set_scalars_kernel(double *scal, double T, double scale)
{
    scal[0] = T;
    scal[1] = scale;
}

cudaError_t launch_set_scalars(tufrg_model *m, double T, double scale)
{
    m->launches++;
    set_scalars_kernel<<<1, 1, 0, m->stream>>>(m->d_scal, T, scale);
    return cudaGetLastError();
}

cudaError_t launch_fermi_shell(tufrg_model *m)
{
    const int n = m->Nk * m->ns;
    fermi_shell_kernel<<<(n + 255) / 256, 256, 0, m->stream>>>(m->d_E, n, m->mu, m->T_reg, m->d_ft,
                                                                 m->precision == TUFRG_FP64 ? nullptr : m->d_ft32);
    return cudaGetLastError();
}

cudaError_t launch_fermi(tufrg_model *m)
{
    if (loops2_supported(m)) return launch_loop_records(m);   // the split two-band kernel reads its own per-k records
    if (m->regulator == TUFRG_REG_MOMENTUM_SHELL) return cudaSuccess;   // tables fixed at init (no Lambda dependence)
    const int n = m->Nk * m->ns;
    FermiEntry32 *ft32 = m->precision == TUFRG_FP64 ? nullptr : m->d_ft32;
    PhaseScope ps(m, PH_FERMI);
    fermi_kernel<<<(n + 255) / 256, 256, 0, m->stream>>>(m->d_E, n, m->mu, m->d_scal, m->d_ft, ft32);
    return cudaGetLastError();
}

cudaError_t launch_density(tufrg_model *m, double mu, double T, double *h_out)
{
    const int n = m->Nk * m->ns;
    const int nb = 256;
    m->launches += 2;
    density_partial<<<nb, 256, 0, m->stream>>>(m->d_E, n, mu, T, m->d_red);
    TUFRG_CUDA_TRY(cudaGetLastError());
    density_final<<<1, 32, 0, m->stream>>>(m->d_red, nb);
    TUFRG_CUDA_TRY(cudaGetLastError());
    double s = 0.0;
    TUFRG_CUDA_TRY(cudaMemcpyAsync(&s, m->d_red + nb, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    TUFRG_CUDA_TRY(cudaStreamSynchronize(m->stream));
    *h_out = s / (double)m->Nk;
    return cudaSuccess;
}

}  // namespace tufrg

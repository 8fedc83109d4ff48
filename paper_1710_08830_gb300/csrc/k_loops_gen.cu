// Loop k-sum for any N_s (used for N_s = 4, 6; the two-band case has dedicated kernels).
//
//   P:  [L^-_{t1t2t3t4}(s)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)} sum_{l1} rho1^{l1}_{t1t3}(s-q) T^{l1}_{t2t4}
//   C:  [L^+_{t1t2t3t4}(u)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)} sum_{l1} rho1^{l1}_{t1t3}(q)   T^{l1}_{t2t4}
//   with rho^l_{tt'} = U_{tl} U*_{t'l},  T^{l1} = sum_{l2} w_{l1 l2} rho2'^{l2},  rho2' = rho2 (P) or conj (C),
//   w the d/dT of the bubbles of Eqs. disc_2a / disc_2b (Eqs. loopminus, loopplus, loop_orbital).
//
// For fixed (s, q) the orbital dressing is the rank-N_s product Y = A B with A[(t1t3)][l] = rho1 and
// B[l][(t2t4)] = T, an N_s^2 x N_s^2 complex matrix.  One CTA owns one transfer momentum; it walks the fine
// mesh column by column; for each batch of KB rows it stages A and B of those k-points in shared memory
// (all threads cooperate: projectors, pair weights, T), then every thread updates its TA x TB tile of
//     W[dy][(t1t3),(t2t4)] += e^{-i ky dy} Y(k)
// for the non-negative dy of the bond differences.  At the end of a column the thread adds
// e^{-i kx dx} W into the FP64 accumulator of its own entries (no other CTA touches this s, so no
// atomics; the order is fixed).  A final kernel writes the other Hermitian half,
// L(-d)[b][a] = conj(L(d)[a][b]), and scales by 1/Nk.
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int GMAXD = 9;
constexpr int GMAXND = 96;
constexpr int KB = 8;          // rows staged per batch

template <typename R> struct FTg;
template <> struct FTg<double> { using t = FermiEntry; };
template <> struct FTg<float> { using t = FermiEntry32; };

template <typename R>
struct GenArgs {
    const typename cpx<R>::t *U;        // [Nk][NS][NS]
    const typename FTg<R>::t *ft;       // [Nk][NS]
    double2 *acc;                       // [Nq][nd][NS^4] FP64 accumulators (zeroed), half plane filled
    int Lq, nc, Lf, nd, ndx, ndyh;
    int dxs[GMAXD], dys[GMAXD];
    int dslot[GMAXD][GMAXD];            // [dxi][dyi] -> delta index (half plane), or -1
    R thr_factor;                       // degenerate-pair switch = thr_factor * T
    const double *Tp;                   // device temperature
};

template <typename C2> __device__ __forceinline__ void cfma(C2 &acc, C2 a, C2 b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ void ldft(const FermiEntry *p, double &e, double &g, double &gp) { e = p->e; g = p->g; gp = p->gp; }
__device__ __forceinline__ void ldft(const FermiEntry32 *p, float &e, float &g, float &gp) { e = p->e; g = p->g; gp = p->gp; }

template <int WHICH, typename R>
__device__ __forceinline__ R gweight(R e1, R g1, R gp1, R e2, R g2, R gp2, R thr)
{
    if (WHICH == 0) {
        const R s = e1 + e2;
        return fabs(s) > thr ? -(g1 + g2) / s : R(-0.5) * (gp1 + gp2);
    } else {
        const R d = e1 - e2;
        return fabs(d) > thr ? (g1 - g2) / d : R(0.5) * (gp1 + gp2);
    }
}

template <typename R, int NS, int TA, int TB, int NDYH, int WHICH>
__global__ void loops_gen_kernel(GenArgs<R> a)
{
    using C2 = typename cpx<R>::t;
    constexpr int NS2 = NS * NS;
    constexpr int GA = NS2 / TA, GB = NS2 / TB;     // thread grid over (a, b) tiles
    constexpr int NT = GA * GB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *ptab = reinterpret_cast<C2 *>(smem_raw);                    // [Lf] e^{-2 pi i n / Lf}
    C2 *sA = ptab + a.Lf;                                          // [KB][NS][NS2] rho1
    C2 *sB = sA + KB * NS * NS2;                                   // [KB][NS][NS2] T
    C2 *sR2 = sB + KB * NS * NS2;                                  // [KB][NS][NS2] rho2'
    R *sW = reinterpret_cast<R *>(sR2 + KB * NS * NS2);            // [KB][NS][NS] pair weights
    const int Lf = a.Lf;
    for (int n = threadIdx.x; n < Lf; n += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)n / (double)Lf, &sn, &cs);
        ptab[n] = mk(R(cs), R(-sn));
    }
    const int s = blockIdx.x;
    const int sx = (s / a.Lq) * a.nc, sy = (s % a.Lq) * a.nc;
    const int ta = threadIdx.x / GB, tb = threadIdx.x % GB;
    const R thr = a.thr_factor * (R)(*a.Tp);
    const bool active = threadIdx.x < NT;
    double2 *acc = a.acc + (size_t)s * a.nd * NS2 * NS2;

    for (int kx = 0; kx < Lf; kx++) {
        C2 W[NDYH][TA][TB];
#pragma unroll
        for (int d = 0; d < NDYH; d++)
#pragma unroll
            for (int i = 0; i < TA; i++)
#pragma unroll
                for (int j = 0; j < TB; j++) W[d][i][j] = mk(R(0), R(0));
        for (int ky0 = 0; ky0 < Lf; ky0 += KB) {
            const int nb = min(KB, Lf - ky0);
            __syncthreads();   // previous batch fully consumed
            // stage projectors of the batch: rho1 (k1 side) into sA, rho2' (k2 side) into sR2
            for (int idx = threadIdx.x; idx < nb * NS * NS2; idx += blockDim.x) {
                const int kb = idx / (NS * NS2), r = idx % (NS * NS2), l = r / NS2, p = r % NS2;
                const int t = p / NS, tp = p % NS;
                const int ky = ky0 + kb;
                const int k1 = WHICH == 0 ? ((sx - kx + Lf) % Lf) * Lf + (sy - ky + Lf) % Lf : kx * Lf + ky;
                const int k2 = WHICH == 0 ? kx * Lf + ky : ((kx - sx + Lf) % Lf) * Lf + (ky - sy + Lf) % Lf;
                const C2 u = a.U[(size_t)k1 * NS2 + t * NS + l], v = a.U[(size_t)k1 * NS2 + tp * NS + l];
                sA[idx] = mk(u.x * v.x + u.y * v.y, u.y * v.x - u.x * v.y);          // u conj(v)
                const C2 x = a.U[(size_t)k2 * NS2 + t * NS + l], y = a.U[(size_t)k2 * NS2 + tp * NS + l];
                sR2[idx] = WHICH == 0 ? mk(x.x * y.x + x.y * y.y, x.y * y.x - x.x * y.y)    // x conj(y)
                                      : mk(x.x * y.x + x.y * y.y, x.x * y.y - x.y * y.x);   // conj(x) y
            }
            for (int idx = threadIdx.x; idx < nb * NS * NS; idx += blockDim.x) {
                const int kb = idx / (NS * NS), l1 = (idx / NS) % NS, l2 = idx % NS;
                const int ky = ky0 + kb;
                const int k1 = WHICH == 0 ? ((sx - kx + Lf) % Lf) * Lf + (sy - ky + Lf) % Lf : kx * Lf + ky;
                const int k2 = WHICH == 0 ? kx * Lf + ky : ((kx - sx + Lf) % Lf) * Lf + (ky - sy + Lf) % Lf;
                R e1, g1, gp1, e2, g2, gp2;
                ldft(&a.ft[(size_t)k1 * NS + l1], e1, g1, gp1);
                ldft(&a.ft[(size_t)k2 * NS + l2], e2, g2, gp2);
                sW[idx] = gweight<WHICH, R>(e1, g1, gp1, e2, g2, gp2, thr);
            }
            __syncthreads();
            // T^{l1}_{p} = sum_l2 w_{l1 l2} rho2'^{l2}_p
            for (int idx = threadIdx.x; idx < nb * NS * NS2; idx += blockDim.x) {
                const int kb = idx / (NS * NS2), l1 = (idx / NS2) % NS, p = idx % NS2;
                C2 t = mk(R(0), R(0));
#pragma unroll
                for (int l2 = 0; l2 < NS; l2++) {
                    const R w = sW[(kb * NS + l1) * NS + l2];
                    const C2 r = sR2[(kb * NS + l2) * NS2 + p];
                    t.x = fma(w, r.x, t.x);
                    t.y = fma(w, r.y, t.y);
                }
                sB[idx] = t;
            }
            __syncthreads();
            if (active) {
                for (int kb = 0; kb < nb; kb++) {
                    const int ky = ky0 + kb;
                    C2 Y[TA][TB];
#pragma unroll
                    for (int i = 0; i < TA; i++)
#pragma unroll
                        for (int j = 0; j < TB; j++) Y[i][j] = mk(R(0), R(0));
#pragma unroll
                    for (int l = 0; l < NS; l++) {
                        C2 av[TA], bv[TB];
#pragma unroll
                        for (int i = 0; i < TA; i++) av[i] = sA[(kb * NS + l) * NS2 + ta * TA + i];
#pragma unroll
                        for (int j = 0; j < TB; j++) bv[j] = sB[(kb * NS + l) * NS2 + tb * TB + j];
#pragma unroll
                        for (int i = 0; i < TA; i++)
#pragma unroll
                            for (int j = 0; j < TB; j++) cfma(Y[i][j], av[i], bv[j]);
                    }
#pragma unroll
                    for (int d = 0; d < NDYH; d++) {
                        if (d >= a.ndyh) break;
                        const C2 ph = ptab[(ky * a.dys[d]) % Lf];
#pragma unroll
                        for (int i = 0; i < TA; i++)
#pragma unroll
                            for (int j = 0; j < TB; j++) cfma(W[d][i][j], ph, Y[i][j]);
                    }
                }
            }
        }
        // add e^{-i kx dx} W into this thread's FP64 accumulators (fixed order, no other writer)
        if (active) {
            for (int xi = 0; xi < a.ndx; xi++) {
                const C2 phx = ptab[((kx * a.dxs[xi]) % Lf + Lf) % Lf];
#pragma unroll
                for (int d = 0; d < NDYH; d++) {
                    if (d >= a.ndyh) break;
                    const int di = a.dslot[xi][d];
                    if (di < 0) continue;
#pragma unroll
                    for (int i = 0; i < TA; i++)
#pragma unroll
                        for (int j = 0; j < TB; j++) {
                            // GEMM indices (t1t3) x (t2t4) -> compact pair indices of the channel
                            const int ga = ta * TA + i, gb = tb * TB + j;
                            const int t1 = ga / NS, t3 = ga % NS, t2 = gb / NS, t4 = gb % NS;
                            const int ra = WHICH == 0 ? t2 * NS + t1 : t1 * NS + t2;
                            const int cb = WHICH == 0 ? t4 * NS + t3 : t3 * NS + t4;
                            const C2 v = W[d][i][j];
                            double2 &o = acc[((size_t)di * NS2 + ra) * NS2 + cb];
                            o.x += (double)phx.x * (double)v.x - (double)phx.y * (double)v.y;
                            o.y += (double)phx.x * (double)v.y + (double)phx.y * (double)v.x;
                        }
                }
            }
        }
    }
}

// Mirror the half plane, L(-d)[b][a] = conj(L(d)[a][b]), and scale by 1/Nk.
__global__ void loops_gen_finish(const double2 *acc, const int *deltas, int nd, int ns2, int Nq, double inv_nk,
                                 const int *partner, double2 *out64, float2 *out32)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t per = (size_t)nd * ns2 * ns2;
    if (idx >= (size_t)Nq * per) return;
    const int s = (int)(idx / per);
    const int r = (int)(idx % per);
    const int d = r / (ns2 * ns2), ab = r % (ns2 * ns2), ia = ab / ns2, ib = ab % ns2;
    const int dx = deltas[2 * d], dy = deltas[2 * d + 1];
    const bool half = dy > 0 || (dy == 0 && dx >= 0);
    double2 v;
    if (half) {
        v = acc[idx];
    } else {
        const double2 w = acc[(size_t)s * per + ((size_t)partner[d] * ns2 + ib) * ns2 + ia];
        v = make_double2(w.x, -w.y);
    }
    v.x *= inv_nk;
    v.y *= inv_nk;
    out64[idx] = v;
    if (out32) out32[idx] = make_float2((float)v.x, (float)v.y);
}

template <typename R, int NS, int TA, int TB, int NDYH, int WHICH>
cudaError_t launch_gen(tufrg_model *m, const GenArgs<R> &a)
{
    using C2 = typename cpx<R>::t;
    constexpr int NS2 = NS * NS;
    constexpr int NT = (NS2 / TA) * (NS2 / TB);
    const int threads = ((NT + 31) / 32) * 32;
    const size_t smem = sizeof(C2) * (m->Lf + 3 * KB * NS * NS2) + sizeof(R) * KB * NS * NS;
    auto kern = loops_gen_kernel<R, NS, TA, TB, NDYH, WHICH>;
    if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhaseScope ps(m, PH_LOOPS);
    kern<<<m->Nq, threads, smem, m->stream>>>(a);
    return cudaGetLastError();
}

template <typename R, int NS, int TA, int TB>
cudaError_t dispatch_gen(tufrg_model *m, const GenArgs<R> &a, int ch)
{
    if (a.ndyh <= 3) return ch == 0 ? launch_gen<R, NS, TA, TB, 3, 0>(m, a) : launch_gen<R, NS, TA, TB, 3, 1>(m, a);
    if (a.ndyh <= 5) return ch == 0 ? launch_gen<R, NS, TA, TB, 5, 0>(m, a) : launch_gen<R, NS, TA, TB, 5, 1>(m, a);
    return cudaErrorNotSupported;
}

template <typename R>
void fill_args(tufrg_model *m, GenArgs<R> &a)
{
    a.Lq = m->Lq; a.nc = m->nc; a.Lf = m->Lf; a.nd = m->nd;
    a.ndx = (int)m->dxs.size();
    int ndyh = 0;
    for (int v : m->dys)
        if (v >= 0) a.dys[ndyh++] = v;
    a.ndyh = ndyh;
    for (int i = 0; i < a.ndx; i++) {
        a.dxs[i] = m->dxs[i];
        for (int j = 0; j < GMAXD; j++) {
            a.dslot[i][j] = -1;
            if (j >= ndyh) continue;
            const int dx = a.dxs[i], dy = a.dys[j];
            if (!(dy > 0 || dx >= 0)) continue;
            for (int d = 0; d < m->nd; d++)
                if (m->deltas[2 * d] == dx && m->deltas[2 * d + 1] == dy) a.dslot[i][j] = d;
        }
    }
}

}  // namespace

bool loops_gen_supported(const tufrg_model *m)
{
    int ndyh = 0;
    for (int v : m->dys) ndyh += v >= 0;
    return (m->ns == 4 || m->ns == 6) && (int)m->dxs.size() <= GMAXD && ndyh <= 5 && m->nd <= GMAXND;
}

cudaError_t launch_loops_gen(tufrg_model *m, int channel_mask)
{
    const size_t ns2 = (size_t)m->ns * m->ns, per = (size_t)m->Nq * m->nd * ns2 * ns2;
    for (int ch = 0; ch < 2; ch++) {
        if (!((channel_mask >> ch) & 1)) continue;
        double2 *acc = reinterpret_cast<double2 *>(m->d_part);
        TUFRG_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(double2) * per, m->stream));
        cudaError_t e;
        if (m->precision == TUFRG_FP64) {
            GenArgs<double> a{};
            a.U = m->d_U; a.ft = m->d_ft; a.acc = acc; a.thr_factor = 1e-5; a.Tp = m->d_scal;
            fill_args(m, a);
            e = m->ns == 6 ? dispatch_gen<double, 6, 2, 3>(m, a, ch) : dispatch_gen<double, 4, 2, 2>(m, a, ch);
        } else {
            GenArgs<float> a{};
            a.U = m->d_U32; a.ft = m->d_ft32; a.acc = acc; a.thr_factor = 1e-2f; a.Tp = m->d_scal;
            fill_args(m, a);
            e = m->ns == 6 ? dispatch_gen<float, 6, 4, 3>(m, a, ch) : dispatch_gen<float, 4, 2, 2>(m, a, ch);
        }
        TUFRG_CUDA_TRY(e);
        PhaseScope ps(m, PH_LOOPRED);
        loops_gen_finish<<<(unsigned)((per + 255) / 256), 256, 0, m->stream>>>(
            acc, m->d_deltas, m->nd, (int)ns2, m->Nq, 1.0 / (double)m->Nk, m->d_dpartner, m->d_Lc + ch * per,
            m->precision == TUFRG_FP64 ? nullptr : m->d_Lc32 + ch * per);
        TUFRG_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace tufrg

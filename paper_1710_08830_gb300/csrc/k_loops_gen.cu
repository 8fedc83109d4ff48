// Loop k-sum for any N_s (used for N_s = 4, 6; the two-band case has dedicated kernels).
//
//   P:  [L^-_{t1t2t3t4}(s)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)} sum_{l1} rho1^{l1}_{t1t3}(s-q) T^{l1}_{t2t4}
//   C:  [L^+_{t1t2t3t4}(u)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)} sum_{l1} rho1^{l1}_{t1t3}(q)   T^{l1}_{t2t4}
//   with rho^l_{tt'} = U_{tl} U*_{t'l},  T^{l1} = sum_{l2} w_{l1 l2} rho2'^{l2},  rho2' = rho2 (P) or conj (C),
//   w the d/dT of the bubbles of Eqs. disc_2a / disc_2b (Eqs. loopminus, loopplus, loop_orbital).
//
// For fixed (s, q) the orbital dressing is the rank-N_s product Y = A B with A[(t1t3)][l] = rho1 and
// B[l][(t2t4)] = T, an N_s^2 x N_s^2 complex matrix.  One CTA owns one transfer momentum; it walks the fine
// mesh column by column in batches of KB rows.  The raw eigenvectors and Fermi entries of a batch arrive in
// shared memory by cp.async while the batch before it is multiplied (two buffers); from them all threads
// form A and B of the batch (projectors, pair weights, T), then every thread updates its TA x TB tile of
//     W[dy][(t1t3),(t2t4)] += e^{-i ky dy} Y(k)
// for the non-negative dy of the bond differences.  At the end of a column the thread adds
// e^{-i kx dx} W into the FP64 accumulator of its own entries (no other CTA touches this s, so no
// atomics; the order is fixed).  A final kernel writes the other Hermitian half,
// L(-d)[b][a] = conj(L(d)[a][b]), and scales by 1/Nk.
#include <cmath>

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
    typename cpx<R>::t *acc;            // [kx range][slot][nd][NS^4] accumulators (zeroed), half plane filled;
                                        // FP64 on the plain path, FP32 on the split path
    int Lq, nc, Lf, nd, ndx, ndyh;
    int dxs[GMAXD], dys[GMAXD];
    int dslot[GMAXD][GMAXD];            // [dxi][dyi] -> delta index (half plane), or -1
    R thr_factor;                       // degenerate-pair switch = thr_factor * T
    const double *Tp;                   // device flow scale (T, or Lambda with the momentum shell)
    R shell_T;                          // > 0: momentum-shell regulator at this temperature (tables hold e, f, h)
    const int *s_list;                  // optional: CTA x sums transfer momentum s_list[x] into accumulator slot x
    int n_slot;                         // momenta per kx range (accumulator slots of one range)
    int kx_len;                         // columns per kx range; CTA y covers [y kx_len, (y + 1) kx_len)
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

// v in [0, 2 L) -> v mod L without a division
__device__ __forceinline__ int wrap1(int v, int L) { return v >= L ? v - L : v; }

// Shared memory of one CTA: two buffers of the raw eigenvectors [2 sides][KB][NS^2] and Fermi entries
// [2 sides][KB][NS] of a batch (side 0: k1, side 1: k2; filled by cp.async one batch ahead), then the phase
// table [Lf], rho1 / T / rho2' [KB][NS][NS^2] each, batch phases [KB][NDYH], pair weights [KB][NS][NS].
template <typename R, int NS>
constexpr size_t gen_raw_bytes()
{
    return 2 * (sizeof(typename cpx<R>::t) * 2 * KB * NS * NS + sizeof(typename FTg<R>::t) * 2 * KB * NS);
}
template <typename R, int NS, int NDYH>
size_t gen_smem(int Lf)
{
    using C2 = typename cpx<R>::t;
    return gen_raw_bytes<R, NS>() + sizeof(C2) * (Lf + 3 * KB * NS * NS * NS + KB * NDYH) + sizeof(R) * KB * NS * NS;
}

template <typename R, int NS, int TA, int TB, int NDYH, int WHICH>
__global__ void loops_gen_kernel(GenArgs<R> a)
{
    using C2 = typename cpx<R>::t;
    constexpr int NS2 = NS * NS;
    constexpr int GA = NS2 / TA, GB = NS2 / TB;     // thread grid over (a, b) tiles
    constexpr int NT = GA * GB;
    using FT = typename FTg<R>::t;
    static_assert(NT >= KB * NDYH, "batch phases are staged by one thread each");
    constexpr int CU = NS2 * (int)sizeof(C2) / 16, CF = NS * (int)sizeof(FT) / 16, CK = CU + CF;
    static_assert(CU * 16 == NS2 * (int)sizeof(C2) && CF * 16 == NS * (int)sizeof(FT), "rows of 16-byte chunks");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *sUr = reinterpret_cast<C2 *>(smem_raw);                     // [2 buffers][2 sides][KB][NS2]
    FT *sFr = reinterpret_cast<FT *>(sUr + 2 * 2 * KB * NS2);       // [2 buffers][2 sides][KB][NS]
    C2 *ptab = reinterpret_cast<C2 *>(smem_raw + gen_raw_bytes<R, NS>());   // [Lf] e^{-2 pi i n / Lf}
    C2 *sA = ptab + a.Lf;                                          // [KB][NS][NS2] rho1
    C2 *sB = sA + KB * NS * NS2;                                   // [KB][NS][NS2] T
    C2 *sR2 = sB + KB * NS * NS2;                                  // [KB][NS][NS2] rho2'
    C2 *sPh = sR2 + KB * NS * NS2;                                 // [KB][NDYH] e^{-i ky dy} of the batch
    R *sW = reinterpret_cast<R *>(sPh + KB * NDYH);                // [KB][NS][NS] pair weights
    const int Lf = a.Lf;
    for (int n = threadIdx.x; n < Lf; n += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)n / (double)Lf, &sn, &cs);
        ptab[n] = mk(R(cs), R(-sn));
    }
    const int s = a.s_list ? a.s_list[blockIdx.x] : blockIdx.x;
    const int sx = (s / a.Lq) * a.nc, sy = (s % a.Lq) * a.nc;
    const int ta = threadIdx.x / GB, tb = threadIdx.x % GB;
    const bool shell = a.shell_T > R(0);
    const R lam = shell ? (R)(*a.Tp) : R(0);
    const R thr = a.thr_factor * (shell ? a.shell_T : (R)(*a.Tp));
    const bool active = threadIdx.x < NT;
    C2 *acc = a.acc + ((size_t)blockIdx.y * a.n_slot + blockIdx.x) * a.nd * NS2 * NS2;
    const int kx_end = min(Lf, (int)(blockIdx.y + 1) * a.kx_len);
    // fine-mesh indices of row ky of column kx: k1 = s - k, k2 = k (P); k1 = k, k2 = k - s (C)
    auto k_of = [&](int side, int kx, int ky) {
        if (side == (WHICH == 0 ? 1 : 0)) return kx * Lf + ky;                      // the point k itself
        return WHICH == 0 ? wrap1(sx - kx + Lf, Lf) * Lf + wrap1(sy - ky + Lf, Lf)  // s - k
                          : wrap1(kx - sx + Lf, Lf) * Lf + wrap1(ky - sy + Lf, Lf); // k - s
    };
    // copies of the raw eigenvectors and Fermi entries of the rows [ky0, ky0 + KB) of column kx into buffer buf
    auto stage_raw = [&](int kx, int ky0, int buf) {
        const int nb = min(KB, Lf - ky0), per_side = nb * CK;
        for (int idx = threadIdx.x; idx < 2 * per_side; idx += blockDim.x) {
            const int side = idx >= per_side, r = idx - side * per_side, kb = r / CK, c = r % CK;
            const int k = k_of(side, kx, ky0 + kb);
            const int slot = (buf * 2 + side) * KB + kb;
            if (c < CU)
                cp_async16(reinterpret_cast<char *>(sUr + (size_t)slot * NS2) + 16 * c,
                           reinterpret_cast<const char *>(a.U + (size_t)k * NS2) + 16 * c);
            else
                cp_async16(reinterpret_cast<char *>(sFr + (size_t)slot * NS) + 16 * (c - CU),
                           reinterpret_cast<const char *>(a.ft + (size_t)k * NS) + 16 * (c - CU));
        }
        cp_async_commit();
    };
    int buf = 0;
    if (blockIdx.y * a.kx_len < kx_end) stage_raw(blockIdx.y * a.kx_len, 0, 0);

    for (int kx = blockIdx.y * a.kx_len; kx < kx_end; kx++) {
        C2 W[NDYH][TA][TB];
#pragma unroll
        for (int d = 0; d < NDYH; d++)
#pragma unroll
            for (int i = 0; i < TA; i++)
#pragma unroll
                for (int j = 0; j < TB; j++) W[d][i][j] = mk(R(0), R(0));
        for (int ky0 = 0; ky0 < Lf; ky0 += KB, buf ^= 1) {
            const int nb = min(KB, Lf - ky0);
            // copies of the next batch (this column's next rows, else the next column's first) go out before
            // this batch is used; the raw buffer they fill was last read before the previous batch's products
            if (ky0 + KB < Lf) stage_raw(kx, ky0 + KB, buf ^ 1);
            else if (kx + 1 < kx_end) stage_raw(kx + 1, 0, buf ^ 1);
            else cp_async_commit();   // an empty group keeps the count of one group in flight
            cp_async_wait<1>();        // this thread's copies of the current batch have landed
            __syncthreads();           // everyone's copies landed; previous batch fully consumed
            const C2 *rU1 = sUr + (size_t)(buf * 2 + 0) * KB * NS2, *rU2 = sUr + (size_t)(buf * 2 + 1) * KB * NS2;
            const FT *rF1 = sFr + (size_t)(buf * 2 + 0) * KB * NS, *rF2 = sFr + (size_t)(buf * 2 + 1) * KB * NS;
            if (threadIdx.x < KB * NDYH) {
                const int kb = threadIdx.x / NDYH, d = threadIdx.x % NDYH;
                if (kb < nb && d < a.ndyh) sPh[threadIdx.x] = ptab[((ky0 + kb) * a.dys[d]) % Lf];
            }
            // stage projectors of the batch: rho1 (k1 side) into sA, rho2' (k2 side) into sR2
            for (int idx = threadIdx.x; idx < nb * NS * NS2; idx += blockDim.x) {
                const int kb = idx / (NS * NS2), r = idx % (NS * NS2), l = r / NS2, p = r % NS2;
                const int t = p / NS, tp = p % NS;
                const C2 u = rU1[kb * NS2 + t * NS + l], v = rU1[kb * NS2 + tp * NS + l];
                sA[idx] = mk(u.x * v.x + u.y * v.y, u.y * v.x - u.x * v.y);          // u conj(v)
                const C2 x = rU2[kb * NS2 + t * NS + l], y = rU2[kb * NS2 + tp * NS + l];
                sR2[idx] = WHICH == 0 ? mk(x.x * y.x + x.y * y.y, x.y * y.x - x.x * y.y)    // x conj(y)
                                      : mk(x.x * y.x + x.y * y.y, x.x * y.y - x.y * y.x);   // conj(x) y
            }
            for (int idx = threadIdx.x; idx < nb * NS * NS; idx += blockDim.x) {
                const int kb = idx / (NS * NS), l1 = (idx / NS) % NS, l2 = idx % NS;
                R e1, g1, gp1, e2, g2, gp2;
                ldft(&rF1[kb * NS + l1], e1, g1, gp1);
                ldft(&rF2[kb * NS + l2], e2, g2, gp2);
                sW[idx] = gen_pair_weight<WHICH, R>(e1, g1, gp1, e2, g2, gp2, thr, lam);
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
                        const C2 ph = sPh[kb * NDYH + d];
#pragma unroll
                        for (int i = 0; i < TA; i++)
#pragma unroll
                            for (int j = 0; j < TB; j++) cfma(W[d][i][j], ph, Y[i][j]);
                    }
                }
            }
        }
        // add e^{-i kx dx} W into this thread's accumulators (fixed order, no other writer)
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
                            C2 &o = acc[((size_t)di * NS2 + ra) * NS2 + cb];
                            o.x += phx.x * v.x - phx.y * v.y;
                            o.y += phx.x * v.y + phx.y * v.x;
                        }
                }
            }
        }
    }
    cp_async_wait<0>();   // nothing in flight at exit (the last group is empty)
}

// re, im += the n values p[c stride] in order c = 0, 1, ... (FP64), eight loads in flight
__device__ __forceinline__ double wide(float v) { return widen_f(v); }
__device__ __forceinline__ double wide(double v) { return v; }
template <typename C2>
__device__ __forceinline__ void sum_ranges(const C2 *p, size_t stride, int n, double &re, double &im)
{
    constexpr int UB = 8;
    int c = 0;
    for (; c + UB <= n; c += UB) {
        C2 w[UB];
#pragma unroll
        for (int j = 0; j < UB; j++) w[j] = p[(size_t)(c + j) * stride];
#pragma unroll
        for (int j = 0; j < UB; j++) {
            re += wide(w[j].x);
            im += wide(w[j].y);
        }
    }
    for (; c < n; c++) {
        const C2 w = p[(size_t)c * stride];
        re += wide(w.x);
        im += wide(w.y);
    }
}

// Mirror the half plane, L(-d)[b][a] = conj(L(d)[a][b]), sum the kx ranges (fixed order) and scale by
// 1/Nk.  Grid: blockIdx.y = momentum, threads over (d, a, b).
template <int NS, typename C2>
__device__ __forceinline__ double2 gen_value(const C2 *acc, size_t chunk_stride, int nchunk, size_t base, int d,
                                             int ia, int ib, const int *deltas, const int *partner)
{
    constexpr int NS2 = NS * NS;
    const int dx = deltas[2 * d], dy = deltas[2 * d + 1];
    const bool half = dy > 0 || (dy == 0 && dx >= 0);
    const size_t o = half ? base + ((size_t)d * NS2 + ia) * NS2 + ib : base + ((size_t)partner[d] * NS2 + ib) * NS2 + ia;
    double re = 0.0, im = 0.0;
    sum_ranges(acc + o, chunk_stride, nchunk, re, im);
    return make_double2(re, half ? im : -im);
}

// blockIdx.y = accumulator slot s (n_slot of them), written at momentum qout[s] (orbit representatives
// only) or at s.
template <int NS, typename C2>
__global__ void loops_gen_finish(const C2 *acc, int nchunk, int n_slot, const int *deltas, int nd, double inv_nk,
                                 const int *partner, const int *qout, double2 *out64, float2 *out32)
{
    constexpr int NS2 = NS * NS, NS4 = NS2 * NS2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd * NS4) return;
    const int s = blockIdx.y, d = t / NS4, ia = (t / NS2) % NS2, ib = t % NS2;
    const size_t per = (size_t)nd * NS4;
    double2 v = gen_value<NS>(acc, (size_t)n_slot * per, nchunk, (size_t)s * per, d, ia, ib, deltas, partner);   // C2 deduced
    v.x *= inv_nk;
    v.y *= inv_nk;
    const size_t o = (size_t)(qout ? qout[s] : s) * per + t;
    if (out64) out64[o] = v;
    if (out32) out32[o] = make_float2((float)v.x, (float)v.y);
}

// Sum of the kx ranges per accumulator slot (fixed order, FP64), before the symmetric gather: the gather
// reads every slot Nq / n_slot times, so it must read one L2-resident value, not one per range from DRAM.
// Grid: (elements / 256, slot).
template <typename C2>
__global__ void loops_gen_chunk_sum(const C2 *acc, int nchunk, int n_slot, int per, double2 *red)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= per) return;
    const size_t o = (size_t)blockIdx.y * per + t, stride = (size_t)n_slot * per;
    double re = 0.0, im = 0.0;
    sum_ranges(acc + o, stride, nchunk, re, im);
    red[o] = make_double2(re, im);
}

// Symmetric variant: blockIdx.y = output momentum q'; qmap[q'] = (accumulator slot of its orbit
// representative, group element e); thread (d', a', b') reads the representative's (d, src a', src b')
// (half plane or its Hermitian mirror) and writes i^(qt[a'] - qt[b']) (conj ? conj(v) : v) / Nk.
template <int NS, typename C2>
__global__ void loops_gen_finish_sym(const C2 *acc, int nchunk, int n_slot, const int *deltas, int nd,
                                     double inv_nk, const int *partner, const int2 *qmap, const SymElem *elem,
                                     const int *dinv, int ch, double2 *out64, float2 *out32)
{
    constexpr int NS2 = NS * NS, NS4 = NS2 * NS2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd * NS4) return;
    const int q2 = blockIdx.y, d2 = t / NS4, a2 = (t / NS2) % NS2, b2 = t % NS2;
    const int2 ie = qmap[q2];
    const SymElem &e = elem[ie.y];
    const size_t per = (size_t)nd * NS4;
    double2 v = gen_value<NS>(acc, (size_t)n_slot * per, nchunk, (size_t)ie.x * per, dinv[ie.y * nd + d2],
                              e.src[ch][a2], e.src[ch][b2], deltas, partner);
    if (e.conj) v.y = -v.y;
    double2 w;
    switch ((e.qt[ch][a2] - e.qt[ch][b2]) & 3) {
    case 0: w = v; break;
    case 1: w = make_double2(-v.y, v.x); break;
    case 2: w = make_double2(-v.x, -v.y); break;
    default: w = make_double2(v.y, -v.x); break;
    }
    w.x *= inv_nk;
    w.y *= inv_nk;
    const size_t o = (size_t)q2 * per + t;
    out64[o] = w;
    if (out32) out32[o] = make_float2((float)w.x, (float)w.y);
}

template <typename R, int NS, int TA, int TB, int NDYH, int WHICH>
cudaError_t launch_gen(tufrg_model *m, const GenArgs<R> &a)
{
    using C2 = typename cpx<R>::t;
    constexpr int NS2 = NS * NS;
    constexpr int NT = (NS2 / TA) * (NS2 / TB);
    const int threads = ((NT + 31) / 32) * 32;
    const size_t smem = gen_smem<R, NS, NDYH>(m->Lf);
    auto kern = loops_gen_kernel<R, NS, TA, TB, NDYH, WHICH>;
    if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhaseScope ps(m, PH_LOOPS);
    kern<<<dim3(a.n_slot, m->gen_chunks), threads, smem, m->stream>>>(a);
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

namespace {

// Resident CTAs per SM of the instantiation the model launches, and the kx ranges per momentum that
// fill the GPU best (at least 4 columns per range).
template <typename R, int NS, int TA, int TB>
int gen_blocks_per_sm(const tufrg_model *m, int ndyh)
{
    constexpr int NS2 = NS * NS, NT = (NS2 / TA) * (NS2 / TB);
    const int threads = ((NT + 31) / 32) * 32;
    int n = 0;
    cudaError_t e = ndyh <= 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, loops_gen_kernel<R, NS, TA, TB, 3, 0>, threads, gen_smem<R, NS, 3>(m->Lf))
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, loops_gen_kernel<R, NS, TA, TB, 5, 0>, threads, gen_smem<R, NS, 5>(m->Lf));
    return (e == cudaSuccess && n > 0) ? n : 1;
}

}  // namespace

size_t gen_red_offset(const tufrg_model *m)
{
    const size_t ns2 = (size_t)m->ns * m->ns;
    return (size_t)m->gen_chunks * m->n_loop_q * m->nd * ns2 * ns2 * sizeof(double2);
}

size_t gen_part_bytes(const tufrg_model *m)
{
    const size_t ns2 = (size_t)m->ns * m->ns;
    return gen_red_offset(m) + (m->sym ? (size_t)m->n_loop_q * m->nd * ns2 * ns2 * sizeof(double2) : 0);
}

int plan_gen_chunks(const tufrg_model *m)
{
    int ndyh = 0;
    for (int v : m->dys) ndyh += v >= 0;
    int per_sm;
    if (m->precision == TUFRG_FP64) per_sm = m->ns == 6 ? gen_blocks_per_sm<double, 6, 2, 3>(m, ndyh) : gen_blocks_per_sm<double, 4, 2, 2>(m, ndyh);
    else per_sm = m->ns == 6 ? gen_blocks_per_sm<float, 6, 4, 3>(m, ndyh) : gen_blocks_per_sm<float, 4, 2, 2>(m, ndyh);
    // minimise (waves) x (columns per range): a grid just over one wave doubles the time
    const long slots = (long)m->sm_count * per_sm;
    int best = 1;
    double best_cost = 1e300;
    for (int c = 1; c <= std::min(16, std::max(1, m->Lf / 4)); c++) {
        const double waves = std::ceil((double)m->n_loop_q * c / (double)slots);
        const double cost = waves * std::ceil((double)m->Lf / c);
        if (cost < best_cost * 0.999) { best_cost = cost; best = c; }
    }
    return best;
}

namespace {

template <typename R>
void fill_chunks(const tufrg_model *m, GenArgs<R> &a)
{
    a.s_list = m->sym ? m->d_loop_list : nullptr;
    a.n_slot = m->sym ? m->n_loop_q : m->Nq;
    a.kx_len = (m->Lf + m->gen_chunks - 1) / m->gen_chunks;
}

}  // namespace

cudaError_t launch_loops_gen(tufrg_model *m, int channel_mask, bool reps_only)
{
    const size_t ns2 = (size_t)m->ns * m->ns, per = (size_t)m->Nq * m->nd * ns2 * ns2;
    const int n_slot = m->sym ? m->n_loop_q : m->Nq;
    const size_t acc_n = (size_t)m->gen_chunks * n_slot * m->nd * ns2 * ns2;
    for (int ch = 0; ch < 2; ch++) {
        if (!((channel_mask >> ch) & 1)) continue;
        const bool fp64 = m->precision == TUFRG_FP64;
        cudaError_t e;
        if (m->loops_tc) {
            // tensor cores: the half-plane sums of every slot are written (not accumulated), one kx range
            e = launch_loops_tc(m, ch, reinterpret_cast<float2 *>(m->d_part));
        } else if (fp64) {
            TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_part, 0, sizeof(double2) * acc_n, m->stream));
            GenArgs<double> a{};
            a.U = m->d_U; a.ft = m->d_ft; a.acc = reinterpret_cast<double2 *>(m->d_part); a.thr_factor = 1e-5; a.Tp = m->d_scal;
            a.shell_T = m->regulator == TUFRG_REG_MOMENTUM_SHELL ? m->T_reg : 0.0;
            fill_args(m, a);
            fill_chunks(m, a);
            e = m->ns == 6 ? dispatch_gen<double, 6, 2, 3>(m, a, ch) : dispatch_gen<double, 4, 2, 2>(m, a, ch);
        } else {
            TUFRG_CUDA_TRY(cudaMemsetAsync(m->d_part, 0, sizeof(float2) * acc_n, m->stream));
            GenArgs<float> a{};
            a.U = m->d_U32; a.ft = m->d_ft32; a.acc = reinterpret_cast<float2 *>(m->d_part); a.thr_factor = 1e-2f; a.Tp = m->d_scal;
            a.shell_T = m->regulator == TUFRG_REG_MOMENTUM_SHELL ? (float)m->T_reg : 0.f;
            fill_args(m, a);
            fill_chunks(m, a);
            e = m->ns == 6 ? dispatch_gen<float, 6, 4, 3>(m, a, ch) : dispatch_gen<float, 4, 2, 2>(m, a, ch);
        }
        TUFRG_CUDA_TRY(e);
        PhaseScope ps(m, PH_LOOPRED);
        double2 *o64 = m->d_Lc + ch * per;
        float2 *o32 = fp64 ? nullptr : m->d_Lc32 + ch * per;
        const int n4 = m->nd * (int)(ns2 * ns2);
        const dim3 grid((n4 + 255) / 256, m->Nq);
        const double inv_nk = 1.0 / (double)m->Nk;
        const double2 *a64 = reinterpret_cast<const double2 *>(m->d_part);
        const float2 *a32 = reinterpret_cast<const float2 *>(m->d_part);
        const int nc = m->gen_chunks;
        auto finish = [&](dim3 g, int n_s, const int *qout, double2 *w64, float2 *w32) {
            if (m->ns == 6 && fp64)
                loops_gen_finish<6><<<g, 256, 0, m->stream>>>(a64, nc, n_s, m->d_deltas, m->nd, inv_nk, m->d_dpartner, qout, w64, w32);
            else if (m->ns == 6)
                loops_gen_finish<6><<<g, 256, 0, m->stream>>>(a32, nc, n_s, m->d_deltas, m->nd, inv_nk, m->d_dpartner, qout, w64, w32);
            else if (fp64)
                loops_gen_finish<4><<<g, 256, 0, m->stream>>>(a64, nc, n_s, m->d_deltas, m->nd, inv_nk, m->d_dpartner, qout, w64, w32);
            else
                loops_gen_finish<4><<<g, 256, 0, m->stream>>>(a32, nc, n_s, m->d_deltas, m->nd, inv_nk, m->d_dpartner, qout, w64, w32);
        };
        if (reps_only) {
            // the representatives at their own momenta; the split path's products read the FP32 loops only
            finish(dim3((n4 + 255) / 256, n_slot), n_slot, m->d_loop_list, fp64 ? o64 : nullptr, o32);
        } else if (m->sym) {
            // the kx ranges summed per representative (same order as the plain finish), then the gather
            double2 *red = reinterpret_cast<double2 *>(static_cast<char *>(m->d_part) + gen_red_offset(m));
            const dim3 g1((n4 + 255) / 256, n_slot);
            if (fp64) loops_gen_chunk_sum<<<g1, 256, 0, m->stream>>>(a64, nc, n_slot, n4, red);
            else loops_gen_chunk_sum<<<g1, 256, 0, m->stream>>>(a32, nc, n_slot, n4, red);
            if (m->ns == 6)
                loops_gen_finish_sym<6><<<grid, 256, 0, m->stream>>>(red, 1, n_slot, m->d_deltas, m->nd, inv_nk, m->d_dpartner,
                                                                     m->d_qmap, m->d_sym_elem, m->d_sym_dinv, ch, o64, o32);
            else
                loops_gen_finish_sym<4><<<grid, 256, 0, m->stream>>>(red, 1, n_slot, m->d_deltas, m->nd, inv_nk, m->d_dpartner,
                                                                     m->d_qmap, m->d_sym_elem, m->d_sym_dinv, ch, o64, o32);
        } else {
            finish(grid, m->Nq, nullptr, o64, o32);
        }
        TUFRG_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace tufrg

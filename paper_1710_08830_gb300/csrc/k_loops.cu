// Single-scale loops in the form-factor x orbital basis by the fine-mesh k-sum.
//
//   P:  [L^-_{t1t2t3t4}(s)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)} sum_{l1 l2}
//         U_{t1l1}(s-q) U*_{t3l1}(s-q) dF^-_{l1l2}/dT U_{t2l2}(q) U*_{t4l2}(q)
//   C:  [L^+_{t1t2t3t4}(u)]_{R1R2} = (1/Nk) sum_q e^{-iq.(R1-R2)} sum_{l1 l2}
//         U_{t1l1}(q) U*_{t3l1}(q) dF^+_{l1l2}/dT U*_{t2l2}(q-u) U_{t4l2}(q-u)
// (Eqs. loopminus / loopplus with the band loops of Eq. def_lmp dressed by Eq. trafo,
//  cf. Eq. loop_orbital; temperature flow, so the weight is d/dT of Eqs. disc_2a/2b.)
//
// GPU design (N_s = 2): one thread per fine-mesh column kx of one transfer momentum;
// it walks a range of rows ky and keeps, in registers,
//     W[dy][ab] = sum_ky e^{-i ky dy} Y(kx, ky)[ab]
// for the non-negative dy of the Hermitian half of the bond differences (the
// other half follows from L(-d)[b][a] = conj(L(d)[a][b])).  The x phase e^{-i kx dx}
// is applied once per column when the warp flushes its sums through shared
// memory into one partial per warp; a second kernel adds the partials in a fixed
// order (deterministic) and writes both halves.  All eigen data stay in L2
// (a few MB), so the kernel is bound by FMA throughput, not by HBM.
#include <algorithm>

#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int NS = 2;
constexpr int NS2 = NS * NS;
constexpr int NS4 = NS2 * NS2;
constexpr int MAXD = 9;          // distinct dx (or dy) values for the bond sets supported
constexpr int WARPS = 2;         // warps per CTA (CTA = 64 columns)

template <typename R> struct FT;
template <> struct FT<double> { using t = FermiEntry; };
template <> struct FT<float> { using t = FermiEntry32; };

template <typename R>
struct LoopArgs {
    const typename cpx<R>::t *U;        // [Nk][NS][NS] (row tau, column band)
    const typename FT<R>::t *ft;        // [Nk][NS]
    typename cpx<R>::t *part;           // [Nq][n_part][ndx][ndyh][NS4]
    int Lq, nc, Lf;
    int ndx, ndyh;
    int dxs[MAXD];                      // distinct dx values
    int dys[MAXD];                      // non-negative dy values (half plane)
    unsigned needed[MAXD];              // bit dyi set if (dx, dy) is a needed half-plane difference
    int ky_chunks, ky_len;
    R thr_factor;                       // degenerate-pair switch = thr_factor * T
    const double *Tp;                   // device flow scale (T, or Lambda with the momentum shell)
    R shell_T;                          // > 0: momentum-shell regulator at this temperature (tables hold e, f, h)
    int which;                          // 0 = P, 1 = C (uniform, also a template arg below)
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
template <typename C2> __device__ __forceinline__ void cfma(C2 &acc, C2 a, C2 b)
{
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ void load_ft(const FermiEntry *p, double &e, double &g, double &gp)
{
    e = p->e; g = p->g; gp = p->gp;
}
__device__ __forceinline__ void load_ft(const FermiEntry32 *p, float &e, float &g, float &gp)
{
    float4 v = *reinterpret_cast<const float4 *>(p);
    e = v.x; g = v.y; gp = v.z;
}

__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }

// d/dT F^-(e1, e2) (P) and d/dT F^+(e1, e2) (C); analytic limit for near-degenerate pairs.  With the
// momentum shell (lam > 0) the entries hold (e, f, h) and the weight is d/dLambda [chi chi] F.
template <int WHICH, typename R>
__device__ __forceinline__ R pair_weight(R e1, R g1, R gp1, R e2, R g2, R gp2, R thr, R lam)
{
    if (lam > R(0)) return shell_weight<WHICH, R>(e1, g1, gp1, e2, g2, gp2, thr, lam);
    if (WHICH == 0) {
        R s = e1 + e2;
        return fabs(s) > thr ? -fdiv(g1 + g2, s) : R(-0.5) * (gp1 + gp2);
    } else {
        R d = e1 - e2;
        return fabs(d) > thr ? fdiv(g1 - g2, d) : R(0.5) * (gp1 + gp2);
    }
}

template <typename R, int NDYH, int NAB, int ABG, int WHICH>
__device__ __forceinline__ void loop_body(const LoopArgs<R> &a, const typename cpx<R>::t *ptab, R *red)
{
    using C2 = typename cpx<R>::t;
    const int s = blockIdx.x;
    const int sx = (s / a.Lq) * a.nc, sy = (s % a.Lq) * a.nc;
    const int Lf = a.Lf;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int kx = blockIdx.y * (32 * WARPS) + threadIdx.x;
    const bool valid = kx < Lf;
    const int kyc = blockIdx.z % a.ky_chunks;   // the ab group is blockIdx.z / ky_chunks
    const bool shell = a.shell_T > R(0);
    const R lam = shell ? (R)(*a.Tp) : R(0);
    const R thr = a.thr_factor * (shell ? a.shell_T : (R)(*a.Tp));
    const int ky0 = kyc * a.ky_len;
    const int ky1 = min(Lf, ky0 + a.ky_len);

    C2 W[NDYH][NAB];
#pragma unroll
    for (int i = 0; i < NDYH; i++)
#pragma unroll
        for (int j = 0; j < NAB; j++) W[i][j] = mk(R(0), R(0));

    if (valid) {
        // fine-mesh column of k1 / k2 (row varies in the loop)
        const int k1x = WHICH == 0 ? (sx - kx + Lf) % Lf : kx;
        const int k2x = WHICH == 0 ? kx : (kx - sx + Lf) % Lf;
        for (int ky = ky0; ky < ky1; ky++) {
            const int k1y = WHICH == 0 ? (sy - ky + Lf) % Lf : ky;
            const int k2y = WHICH == 0 ? ky : (ky - sy + Lf) % Lf;
            const int k1 = k1x * Lf + k1y, k2 = k2x * Lf + k2y;
            C2 U1[NS][NS], U2[NS][NS];
#pragma unroll
            for (int i = 0; i < NS; i++)
#pragma unroll
                for (int l = 0; l < NS; l++) {
                    U1[i][l] = a.U[(size_t)k1 * NS2 + i * NS + l];
                    U2[i][l] = a.U[(size_t)k2 * NS2 + i * NS + l];
                }
            R e1[NS], g1[NS], gp1[NS], e2[NS], g2[NS], gp2[NS];
#pragma unroll
            for (int l = 0; l < NS; l++) {
                load_ft(&a.ft[(size_t)k1 * NS + l], e1[l], g1[l], gp1[l]);
                load_ft(&a.ft[(size_t)k2 * NS + l], e2[l], g2[l], gp2[l]);
            }
            // band projectors: rho1^l_{t t'} = U1_{t l} U1*_{t' l};  rho2 likewise, conjugated for C
            C2 rho1[NS][NS][NS], rho2[NS][NS][NS];
#pragma unroll
            for (int l = 0; l < NS; l++)
#pragma unroll
                for (int t = 0; t < NS; t++)
#pragma unroll
                    for (int tp = 0; tp < NS; tp++) {
                        rho1[l][t][tp] = cmulc(U1[t][l], U1[tp][l]);
                        rho2[l][t][tp] = WHICH == 0 ? cmulc(U2[t][l], U2[tp][l]) : cmulc(U2[tp][l], U2[t][l]);
                    }
            // Tm^{l1}_{t2 t4} = sum_l2 w_{l1 l2} rho2^{l2}_{t2 t4}
            C2 Tm[NS][NS][NS];
#pragma unroll
            for (int l1 = 0; l1 < NS; l1++) {
                R w[NS];
#pragma unroll
                for (int l2 = 0; l2 < NS; l2++)
                    w[l2] = pair_weight<WHICH, R>(e1[l1], g1[l1], gp1[l1], e2[l2], g2[l2], gp2[l2], thr, lam);
#pragma unroll
                for (int t2 = 0; t2 < NS; t2++)
#pragma unroll
                    for (int t4 = 0; t4 < NS; t4++) {
                        C2 acc = mk(R(0), R(0));
#pragma unroll
                        for (int l2 = 0; l2 < NS; l2++) {
                            acc.x = fma(w[l2], rho2[l2][t2][t4].x, acc.x);
                            acc.y = fma(w[l2], rho2[l2][t2][t4].y, acc.y);
                        }
                        Tm[l1][t2][t4] = acc;
                    }
            }
            // this thread's NAB entries of Y[a][b] and their row phases
            C2 ph[NDYH];
#pragma unroll
            for (int i = 0; i < NDYH; i++) ph[i] = ptab[(ky * a.dys[i]) % Lf];
#pragma unroll
            for (int j = 0; j < NAB; j++) {
                const int ab = ABG * NAB + j;
                const int ia = ab / NS2, ib = ab % NS2;
                int t1, t2, t3, t4;
                if (WHICH == 0) { t2 = ia / NS; t1 = ia % NS; t4 = ib / NS; t3 = ib % NS; }
                else            { t1 = ia / NS; t2 = ia % NS; t3 = ib / NS; t4 = ib % NS; }
                C2 y = mk(R(0), R(0));
#pragma unroll
                for (int l1 = 0; l1 < NS; l1++) cfma(y, rho1[l1][t1][t3], Tm[l1][t2][t4]);
#pragma unroll
                for (int i = 0; i < NDYH; i++) cfma(W[i][j], ph[i], y);
            }
        }
    }

    // ---- flush: per distinct dx, multiply by e^{-i kx dx}, sum the warp through smem
    constexpr int NV = 2 * NDYH * NAB;       // reals per lane
    constexpr int PITCH = NV + 1;
    R *buf = red + warp * 32 * PITCH;
    const int n_part = gridDim.y * WARPS * a.ky_chunks;
    const int p = (blockIdx.y * WARPS + warp) * a.ky_chunks + kyc;
    for (int dxi = 0; dxi < a.ndx; dxi++) {
        if (a.needed[dxi] == 0) continue;
        const int n = ((kx * a.dxs[dxi]) % Lf + Lf) % Lf;
        const C2 phx = valid ? ptab[n] : mk(R(0), R(0));
#pragma unroll
        for (int i = 0; i < NDYH; i++)
#pragma unroll
            for (int j = 0; j < NAB; j++) {
                C2 c = cmul(phx, W[i][j]);
                buf[lane * PITCH + 2 * (i * NAB + j)] = c.x;
                buf[lane * PITCH + 2 * (i * NAB + j) + 1] = c.y;
            }
        __syncwarp();
        for (int v = lane; v < NV; v += 32) {
            R acc = R(0);
#pragma unroll 8
            for (int r = 0; r < 32; r++) acc += buf[r * PITCH + v];
            const int i = v / (2 * NAB), j = (v / 2) % NAB, re = v & 1;
            if ((a.needed[dxi] >> i) & 1u) {
                const size_t o = ((((size_t)s * n_part + p) * a.ndx + dxi) * a.ndyh + i) * NS4 + ABG * NAB + j;
                reinterpret_cast<R *>(a.part)[2 * o + re] = acc;
            }
        }
        __syncwarp();
    }
}

template <typename R, int NDYH, int NAB, int WHICH>
__global__ void __launch_bounds__(32 * WARPS) loops_ns2_kernel(LoopArgs<R> a)
{
    using C2 = typename cpx<R>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *ptab = reinterpret_cast<C2 *>(smem_raw);
    R *red = reinterpret_cast<R *>(smem_raw + sizeof(C2) * a.Lf);
    // phase table e^{-2 pi i n / Lf}, n in [0, Lf), computed on the device once per CTA
    for (int n = threadIdx.x; n < a.Lf; n += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)n / (double)a.Lf, &sn, &cs);
        ptab[n] = mk(R(cs), R(-sn));
    }
    __syncthreads();
    constexpr int NABG = NS4 / NAB;
    static_assert(NABG == 1 || NABG == 2 || NABG == 4, "ab groups");
    const int g = blockIdx.z / a.ky_chunks;      // ab group, uniform per CTA
    if (g == 0) loop_body<R, NDYH, NAB, 0, WHICH>(a, ptab, red);
    if (NABG > 1 && g == 1) loop_body<R, NDYH, NAB, (NABG > 1 ? 1 : 0), WHICH>(a, ptab, red);
    if (NABG > 2 && g == 2) loop_body<R, NDYH, NAB, (NABG > 2 ? 2 : 0), WHICH>(a, ptab, red);
    if (NABG > 2 && g == 3) loop_body<R, NDYH, NAB, (NABG > 2 ? 3 : 0), WHICH>(a, ptab, red);
}

// Sum the partials of list position s in a fixed order and scale by 1/Nk; the half-plane partials
// give both Hermitian halves.  The sum runs in the partials' own precision (FP32 on the split path:
// this GPU's FP64 rate would make the reduction, not the memory traffic, its bound), with 16 loads
// in flight per thread (the additions keep their sequential order).
template <typename R>
__device__ __forceinline__ typename cpx<R>::t reduce_one(const typename cpx<R>::t *__restrict__ part, int n_part,
                                                         int ndx, int ndyh, const int *dslot, const int *deltas, int s,
                                                         int d, int ab, R inv_nk)
{
    using C2 = typename cpx<R>::t;
    const int dx = deltas[2 * d], dy = deltas[2 * d + 1];
    const bool half = dy > 0 || (dy == 0 && dx >= 0);
    const int ia = ab / NS2, ib = ab % NS2;
    const int src_ab = half ? ab : ib * NS2 + ia;
    const int slot = dslot[d];   // dxi * ndyh + dyi of the half-plane representative of +-delta
    const size_t stride = (size_t)ndx * ndyh * NS4;
    const C2 *src = part + (size_t)s * n_part * stride + (size_t)slot * NS4 + src_ab;
    R re = 0, im = 0;
    constexpr int UB = 16;
    int p = 0;
    for (; p + UB <= n_part; p += UB) {
        C2 v[UB];
#pragma unroll
        for (int j = 0; j < UB; j++) v[j] = src[(size_t)(p + j) * stride];
#pragma unroll
        for (int j = 0; j < UB; j++) {
            re += v[j].x;
            im += v[j].y;
        }
    }
    for (; p < n_part; p++) {
        const C2 v = src[(size_t)p * stride];
        re += v.x;
        im += v.y;
    }
    return mk(re * inv_nk, (half ? im : -im) * inv_nk);
}

__device__ __forceinline__ double2 to64(double2 v) { return v; }
__device__ __forceinline__ double2 to64(float2 v) { return make_double2(widen_f(v.x), widen_f(v.y)); }

// Grid: blockIdx.y = transfer momentum (list position), blockIdx.z = channel (skipped when not in chmask;
// its partials and outputs are offset by part_cs and out_cs), threads over (d, ab) = t (t >> 4, t & 15):
// no runtime integer division (this GPU issues its conversions to the slow FP64 pipe).  List position s
// is written at momentum qout[s] (orbit representatives only) or at s.
template <typename R>
__global__ void loops_reduce_kernel(const typename cpx<R>::t *__restrict__ part, int n_part, int ndx, int ndyh,
                                    const int *dslot, const int *deltas, int nd, double inv_nk, const int *qout,
                                    double2 *out64, typename cpx<R>::t *out32, const int *skip, int chmask,
                                    size_t part_cs, size_t out_cs)
{
    if (skip && *skip) return;
    const int ch = blockIdx.z;
    if (!((chmask >> ch) & 1)) return;
    part += ch * part_cs;
    if (out64) out64 += ch * out_cs;
    if (out32) out32 += ch * out_cs;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd * NS4) return;
    const int s = blockIdx.y, d = t / NS4, ab = t % NS4;
    const auto v = reduce_one<R>(part, n_part, ndx, ndyh, dslot, deltas, s, d, ab, R(inv_nk));
    const size_t idx = (size_t)(qout ? qout[s] : s) * nd * NS4 + t;
    if (out64) out64[idx] = to64(v);
    if (out32) out32[idx] = v;
}

// Symmetry variant (two bands), gather form: blockIdx.y = output momentum q'; qmap[q'] = (list
// position i of its orbit representative, group element e).  Thread (d', a'b') reads the representative's
// partial sums of d = dinv[e][d'], a = src[a'], b = src[b'] (L2 resident) and writes
// Lc(q')[d'][a'][b'] = i^(qt[a'] - qt[b']) (conj ? conj(v) : v) coalesced (see SymElem).
template <typename C2>
__device__ __forceinline__ C2 quarter_turn(C2 v, int k)
{
    switch (k & 3) {
    case 0: return v;
    case 1: return mk(-v.y, v.x);
    case 2: return mk(-v.x, -v.y);
    default: return mk(v.y, -v.x);
    }
}

template <typename R>
__global__ void loops_reduce_sym_kernel(const typename cpx<R>::t *__restrict__ part, int n_part, int ndx, int ndyh,
                                        const int *dslot, const int *deltas, int nd, const int2 *qmap,
                                        const SymElem *elem, const int *dinv, double inv_nk, double2 *out64,
                                        typename cpx<R>::t *out32, const int *skip, int chmask, size_t part_cs,
                                        size_t out_cs)
{
    if (skip && *skip) return;
    const int ch = blockIdx.z;   // as in loops_reduce_kernel
    if (!((chmask >> ch) & 1)) return;
    part += ch * part_cs;
    out64 += ch * out_cs;
    out32 += ch * out_cs;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nd * NS4) return;
    const int q2 = blockIdx.y, d2 = t / NS4, a2 = (t / NS2) % NS2, b2 = t % NS2;
    const int2 ie = qmap[q2];
    const SymElem &e = elem[ie.y];
    const int d = dinv[ie.y * nd + d2], a = e.src[ch][a2], b = e.src[ch][b2];
    auto v = reduce_one<R>(part, n_part, ndx, ndyh, dslot, deltas, ie.x, d, a * NS2 + b, R(inv_nk));
    if (e.conj) v.y = -v.y;
    const auto w = quarter_turn(v, e.qt[ch][a2] - e.qt[ch][b2]);
    const size_t o = (size_t)q2 * nd * NS4 + t;
    if (out64) out64[o] = to64(w);
    if (out32) out32[o] = w;
}

template <typename R, int NDYH, int NAB, int WHICH>
cudaError_t launch_one(tufrg_model *m, const LoopArgs<R> &a, int n_abg)
{
    dim3 grid(m->Nq, (m->Lf + 32 * WARPS - 1) / (32 * WARPS), a.ky_chunks * n_abg);
    size_t smem = sizeof(typename cpx<R>::t) * m->Lf + sizeof(R) * WARPS * 32 * (2 * NDYH * NAB + 1);
    auto kern = loops_ns2_kernel<R, NDYH, NAB, WHICH>;
    if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhaseScope ps(m, PH_LOOPS);
    kern<<<grid, 32 * WARPS, smem, m->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

LoopPlan plan_loops(const tufrg_model *m)
{
    // Choose the number of ky ranges so that the grid fills whole waves of the
    // SMs; the per-column flush costs about 8 rows of work.
    LoopPlan p{};
    p.kx_per_cta = 32 * WARPS;
    const int ctas_x = (m->Lf + p.kx_per_cta - 1) / p.kx_per_cta;
    const int per_sm = loops2_supported(m) ? loops2_blocks_per_sm(m) : (m->precision == TUFRG_FP64 ? 4 : 6);
    const double slots = (double)m->sm_count * per_sm;
    double best = 1e300;
    int best_c = 1;
    for (int c = 1; c <= 16; c++) {
        const int len = (m->Lf + c - 1) / c;
        if (len < 8) break;
        const double ctas = (double)m->n_loop_q * ctas_x * c * (m->precision == TUFRG_FP64 ? 2 : 1);
        const double waves = std::ceil(ctas / slots);
        const double cost = waves * (len + 8.0);
        if (cost < best * 0.999) { best = cost; best_c = c; }
    }
    p.ky_chunks = best_c;
    p.n_partials = ctas_x * WARPS * best_c;
    return p;
}

std::vector<LoopPlan> loop_plan_candidates(const tufrg_model *m)
{
    // every number of ky ranges per column from 1 to 16 whose ranges keep at least 8 rows
    std::vector<LoopPlan> v;
    const int kx_per_cta = 32 * WARPS, ctas_x = (m->Lf + kx_per_cta - 1) / kx_per_cta;
    for (int c = 1; c <= 16; c++) {
        if ((m->Lf + c - 1) / c < 8) break;
        LoopPlan p{};
        p.kx_per_cta = kx_per_cta;
        p.ky_chunks = c;
        p.n_partials = ctas_x * WARPS * c;
        v.push_back(p);
    }
    return v;
}

// launch shape of the reductions: one row of CTAs per momentum, threads over (d, ab)
static void reduce_shape(const tufrg_model *m, int n_s, dim3 &grid, int &thr)
{
    const int per = m->nd * NS4;
    thr = std::min(1024, (per + 31) / 32 * 32);
    grid = dim3((per + thr - 1) / thr, n_s);
}

cudaError_t launch_loops_reduce_f32(tufrg_model *m, const float2 *part, int n_s, double2 *out64, float2 *out32,
                                    const int *skip)
{
    int ndyh = 0;
    for (int v : m->dys) ndyh += v >= 0;
    dim3 grid;
    int thr;
    reduce_shape(m, n_s, grid, thr);
    PhaseScope ps(m, PH_LOOPRED);
    loops_reduce_kernel<float><<<grid, thr, 0, m->stream>>>(part, m->plan.n_partials, (int)m->dxs.size(), ndyh,
                                                          m->d_dslot, m->d_deltas, m->nd, 1.0 / (double)m->Nk, nullptr,
                                                          out64, out32, skip, 1, 0, 0);
    return cudaGetLastError();
}

cudaError_t launch_loops(tufrg_model *m, int channel_mask, bool reps_only)
{
    if (m->sur) TUFRG_CUDA_TRY(launch_surrogate(m, channel_mask));
    reps_only = reps_only && m->sym;
    if (m->ns != NS) return loops_gen_supported(m) ? launch_loops_gen(m, channel_mask, reps_only) : cudaErrorNotSupported;
    const LoopPlan &pl = m->plan;
    const int ndx = (int)m->dxs.size();
    int ndyh = 0;
    int dys[MAXD];
    for (int v : m->dys)
        if (v >= 0) dys[ndyh++] = v;
    if (loops2_supported(m)) {
        // both channels' k-sums into their own halves of the partial buffer, then one reduction launch
        const int n_s = m->sym ? m->n_loop_q : m->Nq;
        const size_t part_cs = (size_t)n_s * pl.n_partials * ndx * ndyh * NS4, out_cs = (size_t)m->Nq * m->nd * NS4;
        float2 *part = reinterpret_cast<float2 *>(m->d_part);
        const int *skip = m->sur ? m->d_sur_flag : nullptr;
        for (int ch = 0; ch < 2; ch++)
            if ((channel_mask >> ch) & 1)
                TUFRG_CUDA_TRY(launch_loops2_ex(m, ch, m->sym ? m->d_loop_list : nullptr, m->sym ? m->n_loop_q : 0,
                                                part + ch * part_cs, skip));
        dim3 grid;
        int thr;
        reduce_shape(m, reps_only ? m->n_loop_q : m->Nq, grid, thr);
        grid.z = 2;
        const double inv_nk = 1.0 / (double)m->Nk;
        PhaseScope ps(m, PH_LOOPRED);
        if (reps_only)   // the representatives' FP32 loops at their own momenta (what their products read)
            loops_reduce_kernel<float><<<grid, thr, 0, m->stream>>>(part, pl.n_partials, ndx, ndyh, m->d_dslot, m->d_deltas,
                                                                  m->nd, inv_nk, m->d_loop_list, nullptr, m->d_Lc32, skip,
                                                                  channel_mask, part_cs, out_cs);
        else if (m->sym)
            loops_reduce_sym_kernel<float><<<grid, thr, 0, m->stream>>>(
                part, pl.n_partials, ndx, ndyh, m->d_dslot, m->d_deltas, m->nd, m->d_qmap, m->d_sym_elem, m->d_sym_dinv,
                inv_nk, m->d_Lc, m->d_Lc32, skip, channel_mask, part_cs, out_cs);
        else
            loops_reduce_kernel<float><<<grid, thr, 0, m->stream>>>(part, pl.n_partials, ndx, ndyh, m->d_dslot, m->d_deltas,
                                                                  m->nd, inv_nk, nullptr, m->d_Lc, m->d_Lc32, skip,
                                                                  channel_mask, part_cs, out_cs);
        return cudaGetLastError();
    }
    for (int ch = 0; ch < 2; ch++) {
        if (!((channel_mask >> ch) & 1)) continue;
        const double inv_nk = 1.0 / (double)m->Nk;
        if (m->precision == TUFRG_FP64) {
            LoopArgs<double> a{};
            a.U = m->d_U; a.ft = m->d_ft; a.part = reinterpret_cast<double2 *>(m->d_part);
            a.Lq = m->Lq; a.nc = m->nc; a.Lf = m->Lf; a.ndx = ndx; a.ndyh = ndyh;
            for (int i = 0; i < ndx; i++) a.dxs[i] = m->dxs[i];
            for (int i = 0; i < ndyh; i++) a.dys[i] = dys[i];
            for (int i = 0; i < ndx; i++) {
                a.needed[i] = 0;
                for (int j = 0; j < ndyh; j++) {
                    int dx = m->dxs[i], dy = dys[j];
                    bool in = false;
                    for (int d = 0; d < m->nd; d++) in |= (m->deltas[2 * d] == dx && m->deltas[2 * d + 1] == dy);
                    if (in && (dy > 0 || dx >= 0)) a.needed[i] |= 1u << j;
                }
            }
            a.ky_chunks = pl.ky_chunks; a.ky_len = (m->Lf + pl.ky_chunks - 1) / pl.ky_chunks;
            a.thr_factor = 1e-5; a.Tp = m->d_scal; a.which = ch;
            a.shell_T = m->regulator == TUFRG_REG_MOMENTUM_SHELL ? m->T_reg : 0.0;
            cudaError_t e;
            if (ndyh <= 3) e = ch == 0 ? launch_one<double, 3, 8, 0>(m, a, 2) : launch_one<double, 3, 8, 1>(m, a, 2);
            else           e = ch == 0 ? launch_one<double, 5, 4, 0>(m, a, 4) : launch_one<double, 5, 4, 1>(m, a, 4);
            TUFRG_CUDA_TRY(e);
            dim3 grid;
            int thr;
            reduce_shape(m, m->Nq, grid, thr);
            PhaseScope ps(m, PH_LOOPRED);
            loops_reduce_kernel<double><<<grid, thr, 0, m->stream>>>(
                a.part, pl.n_partials, ndx, ndyh, m->d_dslot, m->d_deltas, m->nd, inv_nk, nullptr,
                m->d_Lc + (size_t)ch * m->Nq * m->nd * NS4, nullptr, nullptr, 1, 0, 0);
            TUFRG_CUDA_TRY(cudaGetLastError());
        } else {
            LoopArgs<float> a{};
            a.U = m->d_U32; a.ft = m->d_ft32; a.part = reinterpret_cast<float2 *>(m->d_part);
            a.Lq = m->Lq; a.nc = m->nc; a.Lf = m->Lf; a.ndx = ndx; a.ndyh = ndyh;
            for (int i = 0; i < ndx; i++) a.dxs[i] = m->dxs[i];
            for (int i = 0; i < ndyh; i++) a.dys[i] = dys[i];
            for (int i = 0; i < ndx; i++) {
                a.needed[i] = 0;
                for (int j = 0; j < ndyh; j++) {
                    int dx = m->dxs[i], dy = dys[j];
                    bool in = false;
                    for (int d = 0; d < m->nd; d++) in |= (m->deltas[2 * d] == dx && m->deltas[2 * d + 1] == dy);
                    if (in && (dy > 0 || dx >= 0)) a.needed[i] |= 1u << j;
                }
            }
            a.ky_chunks = pl.ky_chunks; a.ky_len = (m->Lf + pl.ky_chunks - 1) / pl.ky_chunks;
            a.thr_factor = 1e-2f; a.Tp = m->d_scal; a.which = ch;
            a.shell_T = m->regulator == TUFRG_REG_MOMENTUM_SHELL ? (float)m->T_reg : 0.f;
            cudaError_t e;
            if (ndyh <= 3) e = ch == 0 ? launch_one<float, 3, 16, 0>(m, a, 1) : launch_one<float, 3, 16, 1>(m, a, 1);
            else           e = ch == 0 ? launch_one<float, 5, 8, 0>(m, a, 2) : launch_one<float, 5, 8, 1>(m, a, 2);
            TUFRG_CUDA_TRY(e);
            dim3 grid;
            int thr;
            reduce_shape(m, m->Nq, grid, thr);
            PhaseScope ps(m, PH_LOOPRED);
            loops_reduce_kernel<float><<<grid, thr, 0, m->stream>>>(
                a.part, pl.n_partials, ndx, ndyh, m->d_dslot, m->d_deltas, m->nd, inv_nk, nullptr,
                m->d_Lc + (size_t)ch * m->Nq * m->nd * NS4, m->d_Lc32 + (size_t)ch * m->Nq * m->nd * NS4, nullptr, 1, 0, 0);
            TUFRG_CUDA_TRY(cudaGetLastError());
        }
    }
    return cudaSuccess;
}

}  // namespace tufrg

// Multi-orbital loop k-sum on the 5th-generation tensor cores (split path, N_s = 6; Eqs. loopminus, loopplus,
// loop_orbital with the temperature or momentum-shell weights of Eqs. disc_2a, disc_2b, def_lmp).
//
// For a transfer momentum s the compact loop is
//   Lc[Delta][(t1 t3),(t2 t4)] = (1/Nk) sum_k e^{-+ i k.Delta} sum_l rho^l_{t1 t3}(k) T^l_{t2 t4}(s, k)
// with rho^l_{tt'} = U_{tl} U*_{t'l} at the summation point k and T^l = sum_{l2} w_{l l2} rho'^{l2} at its partner:
//   C (u = s):  partner k - u, rho' = conj(U_{t2 l2}) U_{t4 l2}, phase e^{-i k.Delta};
//   P (s):      the sum runs over the first propagator's momentum k' = s - q (a relabelling of the fine mesh),
//               partner s - k', rho' = U_{t2 l2} U*_{t4 l2}, phase e^{-i (s - k').Delta} = e^{-i s.Delta} e^{+i k'.Delta}.
// Written this way the summation point's projectors do not depend on s, so one operand serves several momenta.
// With Delta = (dx, dy) the phase separates; per fine-mesh column kx the sum over ky is one complex GEMM
//   W[(dy, t1 t3)][(s_j, t2 t4)] = sum_{(ky, l)} e^{-+ i ky dy} rho^l_{t1 t3}(kx, ky) * T^l_{t2 t4}(s_j; kx, ky)
// with M = 3 dy x 36 = 108 rows (padded to 128), N = 3 momenta x 36 = 108 columns (padded to 112) and
// K = Lf x 6.  It runs as 3xTF32 (hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor memory), the complex
// product as four real MMA streams (the minus of -Ai Bi by the descriptor's negate-A bit), exactly like the
// V.L.V products.  The x phases e^{-+ i kx dx} are applied afterwards by loops_tc_xsum over the written columns.
//
// The left operand (the phased projectors, four TF32 planes) lives in tensor memory: the producers write it with
// tcgen05.st, and the MMAs read it from there, so shared memory carries only the right operand.
// One persistent CTA per SM walks its (momentum group, column) items.  Warp roles:
//   warps 0-15  producers: per stage (4 ky rows = K of 24) they stage the raw eigenvectors and Fermi entries of
//               the 4 summation points and their 12 partners (cp.async, two stages ahead, four buffers), form
//               the pair weights and row phases, then write the operands' TF32 hi/lo planes: A into tensor memory
//               (lane = row), B into shared memory in the K-major core-matrix layout (each thread one ky row of
//               one row of A and of B);
//   warp 16     TMEM allocation and the MMA issuer (one thread): 36 MMAs per stage;
//   warps 17-20 epilogue: tensor memory -> W in global memory (coalesced, row index fastest).
// Two stage buffers (mbarriers full / empty) so operand generation and MMAs overlap; one tensor-memory accumulator
// (mbarriers acc_full / acc_empty): the next column's MMAs start once the epilogue has read the previous one.  Every wait is bounded; on time-out
// the kernel raises the error flag, every role stops, the MMAs in flight are waited for (bounded), the
// cp.async copies drained, and the tensor memory is freed.
#include <algorithm>
#include <cmath>

#include "tc_common.cuh"
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int NS = 6, NS2 = 36, NS4 = NS2 * NS2;
constexpr int GRP = 3;                       // transfer momenta per item (column blocks of B)
constexpr int NDYM = 3;                      // non-negative y components of the bond differences (row blocks of A)
constexpr int ROWS = NDYM * NS2;             // 108 rows used
constexpr int COLS = GRP * NS2;              // 108 columns used
constexpr int TM = 128;                      // MMA M
constexpr int TN = 112;                      // MMA N: COLS padded to a multiple of 16
constexpr int KB = 4;                        // ky rows per stage
constexpr int KST = KB * NS;                 // K per stage: 24 = three MMA K-steps of 8
constexpr int NPROD = 512;                   // producer threads, warps 0-15: thread (ky row kb, operand row r)
constexpr int MMA_WARP = 16;                 // warps 17-20: epilogue
constexpr int NTHREADS = 21 * 32;
constexpr int NRAW = 4;                      // raw staging buffers (stage n + 2 is fetched while n is formed)
constexpr unsigned B_PLANE = TN * KST * 4;   // bytes per plane and stage of the right operand (shared memory)
constexpr unsigned STAGE_BYTES = 4 * B_PLANE;   // planes: Re hi, Re lo, Im hi, Im lo
// tensor memory: accumulator Re at [0, TN), Im at [128, 128 + TN); left operand of stage b at 256 + 128 b, plane p
// at + 32 p (K = 24 columns used)
constexpr unsigned ACC_IM = 128, A_COL0 = 256, A_STAGE_COLS = 128, A_PLANE_COLS = 32;
constexpr int NPTS = KB * (1 + GRP);         // raw points per stage: 4 summation points, then [j][kb] partners
constexpr int CU = NS2 * 8 / 16, CF = NS * 16 / 16, CP = CU + CF;   // 16-byte chunks per point: U, Fermi entries
constexpr unsigned RAW_U = NPTS * NS2 * 8, RAW_BYTES = RAW_U + NPTS * NS * 16;
constexpr unsigned TMEM_COLS = 512;
constexpr unsigned SW_BYTES = GRP * KB * NS * 8 * 4;         // pair weights, rows padded to 8
constexpr size_t SMEM_BYTES = 2 * (size_t)STAGE_BYTES + NRAW * (size_t)RAW_BYTES + SW_BYTES + KB * NDYM * 8 + 4 * NPTS * 4;

struct LtArgs {
    const float2 *U;            // [Nk][NS][NS] eigenvectors (row orbital, column band), FP32
    const FermiEntry32 *ft;     // [Nk][NS] (e, g, g') at the flow scale, or (e, f, h) with the momentum shell
    float2 *W;                  // [n_groups][Lf][COLS][ROWS] column sums
    const int *s_list;          // slot -> transfer momentum (null: the slot is the momentum)
    int n_slot, n_groups, n_items;
    int Lq, nc, Lf, spc;        // spc: stages per column
    int ndyh;
    int dys[NDYM];
    const double *Tp;           // device flow scale
    float thr_factor, shell_T;
    int *err;
};

__device__ __forceinline__ int wrapm(int v, int L)
{
    v %= L;
    return v < 0 ? v + L : v;
}


// six consecutive complex values from shared memory (16-byte aligned) as three 16-byte loads
__device__ __forceinline__ void ld6(const float2 *p, float2 (&v)[NS])
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float4 t = q[i];
        v[2 * i] = make_float2(t.x, t.y);
        v[2 * i + 1] = make_float2(t.z, t.w);
    }
}

// the loop weight of one band pair (gen_pair_weight) with the FP32 fast division of the split two-band kernel
template <int WHICH>
__device__ __forceinline__ float tc_pair_weight(float e1, float g1, float gp1, float e2, float g2, float gp2, float thr, float lam)
{
    if (lam > 0.f) return shell_weight<WHICH, float>(e1, g1, gp1, e2, g2, gp2, thr, lam);
    if (WHICH == 0) {
        const float s = e1 + e2;
        return fabsf(s) > thr ? -__fdividef(g1 + g2, s) : -0.5f * (gp1 + gp2);
    }
    const float d = e1 - e2;
    return fabsf(d) > thr ? __fdividef(g1 - g2, d) : 0.5f * (gp1 + gp2);
}

// TF32 part of x by truncation (the 13 low mantissa bits cleared; one logic operation): x - hi is exact and below
// 2^-10 |x|, so hi + lo keeps FP32 accuracy through the three products of 3xTF32
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

// writes 4 consecutive K values of one row of a plane group (Re hi, Re lo, Im hi, Im lo) as TF32 hi / lo parts
__device__ __forceinline__ void put4(float *planes, unsigned plane_floats, int off, float2 v0, float2 v1, float2 v2, float2 v3)
{
    float4 h, l;
    h = make_float4(tf32_trunc(v0.x), tf32_trunc(v1.x), tf32_trunc(v2.x), tf32_trunc(v3.x));
    l = make_float4(v0.x - h.x, v1.x - h.y, v2.x - h.z, v3.x - h.w);
    *reinterpret_cast<float4 *>(planes + 0 * plane_floats + off) = h;
    *reinterpret_cast<float4 *>(planes + 1 * plane_floats + off) = l;
    h = make_float4(tf32_trunc(v0.y), tf32_trunc(v1.y), tf32_trunc(v2.y), tf32_trunc(v3.y));
    l = make_float4(v0.y - h.x, v1.y - h.y, v2.y - h.z, v3.y - h.w);
    *reinterpret_cast<float4 *>(planes + 2 * plane_floats + off) = h;
    *reinterpret_cast<float4 *>(planes + 3 * plane_floats + off) = l;
}

// two consecutive K values (an even k) of one row
__device__ __forceinline__ void put2(float *planes, unsigned plane_floats, int off, float2 v0, float2 v1)
{
    float2 h, l;
    h = make_float2(tf32_trunc(v0.x), tf32_trunc(v1.x));
    l = make_float2(v0.x - h.x, v1.x - h.y);
    *reinterpret_cast<float2 *>(planes + 0 * plane_floats + off) = h;
    *reinterpret_cast<float2 *>(planes + 1 * plane_floats + off) = l;
    h = make_float2(tf32_trunc(v0.y), tf32_trunc(v1.y));
    l = make_float2(v0.y - h.x, v1.y - h.y);
    *reinterpret_cast<float2 *>(planes + 2 * plane_floats + off) = h;
    *reinterpret_cast<float2 *>(planes + 3 * plane_floats + off) = l;
}

// the six K values kb * 6 + l (l = 0..5) of row r of an R-row operand: 4 + 2 or 2 + 4 along the 4-wide groups
__device__ __forceinline__ void put6(float *planes, unsigned plane_floats, int r, int kb, int R, const float2 (&v)[NS])
{
    const int k0 = 6 * kb;
    if ((kb & 1) == 0) {
        put4(planes, plane_floats, tc::core_off(r, k0, R), v[0], v[1], v[2], v[3]);
        put2(planes, plane_floats, tc::core_off(r, k0 + 4, R), v[4], v[5]);
    } else {
        put2(planes, plane_floats, tc::core_off(r, k0, R), v[0], v[1]);
        put4(planes, plane_floats, tc::core_off(r, k0 + 2, R), v[2], v[3], v[4], v[5]);
    }
}

// the six K values kb * 6 + l of this lane's row of the left operand into tensor memory: four planes (Re hi, Re lo,
// Im hi, Im lo, truncation split) at columns col0 + 32 p + 6 kb + l, as a 4 + 2 (kb even) or 2 + 4 (kb odd) column
// split so that every store starts at a multiple of its width; warp-collective (every lane of the warp)
__device__ __forceinline__ void put6_tmem(unsigned col0, int kb, const float2 (&v)[NS])
{
    const unsigned c = col0 + 6 * kb;
    const bool even = (kb & 1) == 0;
#pragma unroll
    for (int p = 0; p < 4; p++) {
        float t[NS];
#pragma unroll
        for (int l = 0; l < NS; l++) {
            const float x = p < 2 ? v[l].x : v[l].y;
            t[l] = (p & 1) ? x - tf32_trunc(x) : tf32_trunc(x);
        }
        const unsigned cp = c + p * A_PLANE_COLS;
        if (even) {
            tc::tmem_st4(cp, t[0], t[1], t[2], t[3]);
            tc::tmem_st2(cp + 4u, t[4], t[5]);
        } else {
            tc::tmem_st2(cp, t[0], t[1]);
            tc::tmem_st4(cp + 2u, t[2], t[3], t[4], t[5]);
        }
    }
}

__device__ __forceinline__ void bar_producers() { asm volatile("bar.sync 1, %0;" ::"n"(NPROD) : "memory"); }

template <int WHICH>
__global__ void __launch_bounds__(NTHREADS, 1) loops_tc_kernel(LtArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // stage buffer b at smem + b STAGE_BYTES, raw buffer b at smem + 2 STAGE_BYTES + b RAW_BYTES
    auto stage = [&](int b) { return smem + (size_t)b * STAGE_BYTES; };
    auto raw = [&](int b) { return smem + 2 * (size_t)STAGE_BYTES + (size_t)b * RAW_BYTES; };
    float *sW = reinterpret_cast<float *>(smem + 2 * STAGE_BYTES + NRAW * RAW_BYTES);   // [GRP][KB][NS][8]
    float2 *sPh = reinterpret_cast<float2 *>(smem + 2 * STAGE_BYTES + NRAW * RAW_BYTES + SW_BYTES);   // [KB][NDYM]
    int *sPt = reinterpret_cast<int *>(sPh + KB * NDYM);                                   // [4][NPTS]
    __shared__ __align__(8) unsigned long long full[2], empty[2], accf[2], acce[2], done;
    __shared__ unsigned tmem_base;
    __shared__ int abort_flag, stop;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // kernel arguments used inside the lambdas below, copied to registers (no local copy of the struct)
    const int Lf = a.Lf, Lq = a.Lq, nc = a.nc, spc = a.spc, n_slot = a.n_slot;
    const int *const s_list = a.s_list;
    const float2 *const Ug = a.U;
    const FermiEntry32 *const Fg = a.ft;

    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_base)),
                     "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(tc::smem_u32(&full[b]), NPROD);
            tc::mbar_init(tc::smem_u32(&empty[b]), 1);
            tc::mbar_init(tc::smem_u32(&accf[b]), 1);
            tc::mbar_init(tc::smem_u32(&acce[b]), 128);
        }
        tc::mbar_init(tc::smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
        stop = 0;
    }
    // padding rows of B (108..111) are zero in both stage buffers for the whole kernel (the padding lanes of A are
    // written as zeros with every stage)
    for (int i = tid; i < 2 * 4 * (TN - COLS) * KST; i += NTHREADS) {
        const int per_buf = 4 * (TN - COLS) * KST, b = i / per_buf, r0 = i % per_buf;
        const int plane = r0 / ((TN - COLS) * KST), r1 = r0 % ((TN - COLS) * KST);
        const int row = r1 / KST, k = r1 % KST;
        float *base = reinterpret_cast<float *>(stage(b));
        base[plane * (B_PLANE / 4) + tc::core_off(COLS + row, k, TN)] = 0.f;
    }
    tc::fence_smem_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tmem = tmem_base;
    const int my_items = a.n_items > (int)blockIdx.x ? (a.n_items - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int n_stages = my_items * a.spc;

    if (warp < MMA_WARP) {
        // ------------------------------------------------------------------ producers
        const bool shell = a.shell_T > 0.f;
        const float lam = shell ? (float)(*a.Tp) : 0.f;
        const float thr = a.thr_factor * (shell ? a.shell_T : (float)(*a.Tp));
        const int kb = tid >> 7, r = tid & 127;   // ky row of the stage (warp-uniform) and operand row
        // fine-mesh index of raw point p of stage n (-1 when its row or momentum does not exist); evaluated once
        // per stage and point, three stages ahead, into sPt[n % 4]
        auto point = [&](int n, int p) {
            const int item = (int)blockIdx.x + (n / spc) * (int)gridDim.x, st = n % spc;
            const int g = item / Lf, kx = item % Lf;
            const int pk = p & (KB - 1), ky = st * KB + pk;
            if (n >= n_stages || ky >= Lf) return -1;
            if (p < KB) return kx * Lf + ky;
            const int slot = g * GRP + (p - KB) / KB;
            if (slot >= n_slot) return -1;
            const int s = s_list ? s_list[slot] : slot;
            const int sx = (s / Lq) * nc, sy = (s % Lq) * nc;
            return WHICH == 0 ? wrapm(sx - kx, Lf) * Lf + wrapm(sy - ky, Lf) : wrapm(kx - sx, Lf) * Lf + wrapm(ky - sy, Lf);
        };
        auto fetch = [&](int n) {
            if (n < n_stages) {
                unsigned char *rb = raw(n % NRAW);
                const int *pts = sPt + (n & 3) * NPTS;
                for (int i = tid; i < NPTS * CP; i += NPROD) {
                    const int p = i / CP, c = i % CP, k = pts[p];
                    if (k < 0) {   // a row or momentum that does not exist: zeros (no operand value then depends on it)
                        unsigned char *d = c < CU ? rb + (size_t)p * NS2 * 8 + 16 * c : rb + RAW_U + (size_t)p * NS * 16 + 16 * (c - CU);
                        *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
                        continue;
                    }
                    if (c < CU) cp_async16(rb + (size_t)p * NS2 * 8 + 16 * c, reinterpret_cast<const char *>(Ug + (size_t)k * NS2) + 16 * c);
                    else cp_async16(rb + RAW_U + (size_t)p * NS * 16 + 16 * (c - CU),
                                    reinterpret_cast<const char *>(Fg + (size_t)k * NS) + 16 * (c - CU));
                }
            }
            cp_async_commit();
        };
        if (tid < 3 * NPTS) sPt[tid] = point(tid / NPTS, tid % NPTS);
        bar_producers();
        fetch(0);
        fetch(1);
        int item = (int)blockIdx.x, st = 0;   // item and stage within the column of stage n
        for (int n = 0; n < n_stages; n++) {
            const int g = item / Lf;
            const int buf = n & 1;
            // raw buffer (n + 2) % 4 was last read by stage n - 2, which every producer has finished
            fetch(n + 2);
            cp_async_wait<2>();
            bar_producers();          // raw data of stage n landed; stage n - 1 fully formed (sW, sPh, sPt free)
            const float2 *rU = reinterpret_cast<const float2 *>(raw(n % NRAW));
            const FermiEntry32 *rF = reinterpret_cast<const FermiEntry32 *>(raw(n % NRAW) + RAW_U);
            // pair weights [j][kb][l1][8] (rows padded to 8), the row phases [kb][dy] and the points of stage n + 3
            if (tid < GRP * KB * NS * NS) {
                const int i = tid, j = i / (KB * NS * NS), wk = (i / (NS * NS)) % KB, l1 = (i / NS) % NS, l2 = i % NS;
                const int pp = KB + j * KB + wk;
                float w = 0.f;
                if (st * KB + wk < Lf && g * GRP + j < n_slot) {
                    const FermiEntry32 f1 = rF[wk * NS + l1], f2 = rF[pp * NS + l2];
                    w = tc_pair_weight<WHICH>(f1.e, f1.g, f1.gp, f2.e, f2.g, f2.gp, thr, lam);
                }
                sW[((j * KB + wk) * NS + l1) * 8 + l2] = w;
            } else if (tid >= NPROD - KB * NDYM) {
                const int i = tid - (NPROD - KB * NDYM), pk = i / NDYM, dyi = i % NDYM, ky = st * KB + pk;
                const int dyv = dyi == 0 ? a.dys[0] : dyi == 1 ? a.dys[1] : a.dys[2];
                float sn = 0.f, cs = 0.f;
                if (ky < Lf && dyi < a.ndyh) sincospif(2.0f * (float)wrapm(ky * dyv, Lf) / (float)Lf, &sn, &cs);
                sPh[i] = make_float2(cs, WHICH == 0 ? sn : -sn);   // zero for missing rows and y components
            } else if (tid >= NPROD - KB * NDYM - NPTS) {
                const int p = tid - (NPROD - KB * NDYM - NPTS);
                sPt[((n + 3) & 3) * NPTS + p] = point(n + 3, p);
            }
            if (tid == 0) stop = *(volatile int *)&abort_flag;
            bar_producers();
            if (stop) break;   // every producer reads the same value: they leave the loop together
            float *pb = reinterpret_cast<float *>(stage(buf));
            float2 va[NS];
#pragma unroll
            for (int l = 0; l < NS; l++) va[l] = make_float2(0.f, 0.f);   // the padding lanes of A (rows 108..127)
            if (r < ROWS) {
                // A row r = (dy, t1 t3): e^{-+ i ky dy} rho^l_{t1 t3}(k) at K = kb * 6 + l (zero for a missing row: the
                // phase is zero there, and so are the raw values of a point that does not exist)
                const int dyi = r / NS2, ab = r % NS2, t1 = ab / NS, t3 = ab % NS;
                const float2 ph = sPh[kb * NDYM + dyi];
                float2 u[NS], w[NS];
                ld6(rU + kb * NS2 + t1 * NS, u);
                ld6(rU + kb * NS2 + t3 * NS, w);
#pragma unroll
                for (int l = 0; l < NS; l++) {
                    // rho = u conj(w) = u w.x + (u.y, -u.x) w.y;  ph rho = rho ph.x + (-rho.y, rho.x) ph.y
                    const float2 rho = __ffma2_rn(make_float2(u[l].y, -u[l].x), make_float2(w[l].y, w[l].y),
                                                  __fmul2_rn(u[l], make_float2(w[l].x, w[l].x)));
                    va[l] = __ffma2_rn(make_float2(-rho.y, rho.x), make_float2(ph.y, ph.y),
                                       __fmul2_rn(rho, make_float2(ph.x, ph.x)));
                }
            }
            // the MMAs that read this stage (tensor-memory A, shared-memory B) two stages ago must be complete before
            // it is overwritten
            int ok = 1;
            if (n >= 2 && lane == 0)
                ok = tc::mbar_wait_or_abort(tc::smem_u32(&empty[buf]), ((n >> 1) - 1) & 1, &abort_flag) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                // raise the flag and keep the producers in step: all of them leave at the next stage's check
                if (lane == 0) {
                    atomicExch(&abort_flag, 1);
                    atomicExch(a.err, 1);
                }
            } else {
                tc::fence_after();
                // A: this warp's 32 lanes (rows) of the stage's tensor-memory columns, every lane (also padding)
                put6_tmem(tmem + ((unsigned)((warp & 3) * 32) << 16) + A_COL0 + buf * A_STAGE_COLS, kb, va);
                if (r < ROWS) {
                    // B row r = (s_j, t2 t4): T^l_{t2 t4} = sum_l2 w_{l l2} rho'^{l2}_{t2 t4} at K = kb * 6 + l (the
                    // weights of a missing row or momentum are zero)
                    const int j = r / NS2, cd = r % NS2, t2 = cd / NS, t4 = cd % NS, pp = KB + j * KB + kb;
                    float2 x[NS], y[NS], vb[NS];
                    ld6(rU + pp * NS2 + t2 * NS, x);
                    ld6(rU + pp * NS2 + t4 * NS, y);
                    float2 rho[NS];
#pragma unroll
                    for (int l2 = 0; l2 < NS; l2++)
                        rho[l2] = WHICH == 0
                                      // x conj(y) = x y.x + (x.y, -x.x) y.y
                                      ? __ffma2_rn(make_float2(x[l2].y, -x[l2].x), make_float2(y[l2].y, y[l2].y),
                                                   __fmul2_rn(x[l2], make_float2(y[l2].x, y[l2].x)))
                                      // conj(x) y = y x.x + (y.y, -y.x) x.y
                                      : __ffma2_rn(make_float2(y[l2].y, -y[l2].x), make_float2(x[l2].y, x[l2].y),
                                                   __fmul2_rn(y[l2], make_float2(x[l2].x, x[l2].x)));
#pragma unroll
                    for (int l1 = 0; l1 < NS; l1++) {
                        const float4 w0 = *reinterpret_cast<const float4 *>(sW + ((j * KB + kb) * NS + l1) * 8);
                        const float2 w1 = *reinterpret_cast<const float2 *>(sW + ((j * KB + kb) * NS + l1) * 8 + 4);
                        const float wl[NS] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
                        float2 t = __fmul2_rn(make_float2(wl[0], wl[0]), rho[0]);
#pragma unroll
                        for (int l2 = 1; l2 < NS; l2++) t = __ffma2_rn(make_float2(wl[l2], wl[l2]), rho[l2], t);
                        vb[l1] = t;
                    }
                    put6(pb, B_PLANE / 4, r, kb, TN, vb);
                }
                tc::tmem_wait_st();
                tc::fence_smem_async();
                tc::fence_before();
                tc::mbar_arrive(tc::smem_u32(&full[buf]));
            }
            if (++st == spc) {
                st = 0;
                item += (int)gridDim.x;
            }
        }
        cp_async_wait<0>();
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const unsigned id = tc::idesc_tf32(TM, TN, false), idn = tc::idesc_tf32(TM, TN, true);
            bool ok = true;
            int n = 0;
            for (int col = 0; col < my_items && ok; col++) {
                // the accumulator must have been read by the epilogue of the previous column
                if (col >= 1 && !tc::mbar_wait_or_abort(tc::smem_u32(&acce[0]), (col - 1) & 1, &abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                const unsigned tr = tmem, ti = tmem + ACC_IM;
                for (int st = 0; st < a.spc; st++, n++) {
                    const int b = n & 1;
                    if (!tc::mbar_wait_or_abort(tc::smem_u32(&full[b]), (n >> 1) & 1, &abort_flag)) { ok = false; break; }
                    tc::fence_after();
                    const unsigned sb = tc::smem_u32(stage(b)), ta = tmem + A_COL0 + b * A_STAGE_COLS;
#pragma unroll
                    for (int kk = 0; kk < KST / 8; kk++) {
                        const unsigned bo = kk * 2 * (TN / 8) * 128;
                        // A planes in tensor memory: K-step kk = 8 columns of each plane
                        const unsigned arh = ta + 0 * A_PLANE_COLS + 8 * kk, arl = ta + 1 * A_PLANE_COLS + 8 * kk;
                        const unsigned aih = ta + 2 * A_PLANE_COLS + 8 * kk, ail = ta + 3 * A_PLANE_COLS + 8 * kk;
                        const unsigned long long brh = tc::smem_desc(sb + 0 * B_PLANE + bo, TN), brl = tc::smem_desc(sb + 1 * B_PLANE + bo, TN);
                        const unsigned long long bih = tc::smem_desc(sb + 2 * B_PLANE + bo, TN), bil = tc::smem_desc(sb + 3 * B_PLANE + bo, TN);
                        const unsigned first = (st == 0 && kk == 0) ? 0u : 1u;
                        tc::mma_tf32_ta(tr, arh, brh, id, first);  tc::mma_tf32_ta(tr, arh, brl, id, 1u);  tc::mma_tf32_ta(tr, arl, brh, id, 1u);
                        tc::mma_tf32_ta(tr, aih, bih, idn, 1u);    tc::mma_tf32_ta(tr, aih, bil, idn, 1u); tc::mma_tf32_ta(tr, ail, bih, idn, 1u);
                        tc::mma_tf32_ta(ti, arh, bih, id, first);  tc::mma_tf32_ta(ti, arh, bil, id, 1u);  tc::mma_tf32_ta(ti, arl, bih, id, 1u);
                        tc::mma_tf32_ta(ti, aih, brh, id, 1u);     tc::mma_tf32_ta(ti, aih, brl, id, 1u);  tc::mma_tf32_ta(ti, ail, brh, id, 1u);
                    }
                    tc::commit(tc::smem_u32(&empty[b]));
                }
                if (ok) tc::commit(tc::smem_u32(&accf[0]));
            }
            if (!ok) {
                atomicExch(&abort_flag, 1);
                atomicExch(a.err, 1);
            }
            tc::commit(tc::smem_u32(&done));   // completion of every MMA issued above
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ epilogue: tensor memory -> W
        const int qw = warp & 3, row = qw * 32 + lane;
        const unsigned lane_off = (unsigned)(qw * 32) << 16;
        for (int col = 0; col < my_items; col++) {
            int ok = 1;
            if (lane == 0) ok = tc::mbar_wait_or_abort(tc::smem_u32(&accf[0]), col & 1, &abort_flag) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicExch(&abort_flag, 1);
                    atomicExch(a.err, 1);
                }
                break;
            }
            tc::fence_after();
            const int item = (int)blockIdx.x + col * (int)gridDim.x, g = item / Lf, kx = item % Lf;
            float2 *Wc = a.W + ((size_t)g * Lf + kx) * COLS * ROWS;
            for (int c0 = 0; c0 < TN; c0 += 8) {
                unsigned vr[8], vi[8];
                tc::tmem_ld8(tmem + lane_off + (unsigned)c0, vr);
                tc::tmem_ld8(tmem + lane_off + ACC_IM + (unsigned)c0, vi);
                tc::tmem_wait_ld();
                if (row < ROWS) {
#pragma unroll
                    for (int jj = 0; jj < 8; jj++) {
                        const int j = c0 + jj;
                        if (j < COLS) Wc[(size_t)j * ROWS + row] = make_float2(__uint_as_float(vr[jj]), __uint_as_float(vi[jj]));
                    }
                }
            }
            tc::fence_before();
            tc::mbar_arrive(tc::smem_u32(&acce[0]));
        }
    }
    __syncthreads();
    if (tid == MMA_WARP * 32) (void)tc::mbar_wait(tc::smem_u32(&done), 0);   // bounded; the MMAs read shared memory
    tc::fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc::fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

struct XsArgs {
    const float2 *W;            // [n_groups][Lf][COLS][ROWS]
    float2 *acc;                // [n_slot][nd][NS2][NS2] half-plane entries written
    const int *s_list;
    int n_slot, n_groups, Lq, nc, Lf, nd, ndx, ndyh;
    int dxs[9], dys[NDYM];
    int dslot[9][NDYM];         // [dx index][dy index] -> delta index of the half plane, or -1
};

// x phases and the P-channel momentum phase: acc[slot][d][ra][cb] = sum_kx e^{-+ i kx dx} W[g][kx][j][r]
// (times e^{-i s.Delta} for P), one thread per (group, column j, row r), r fastest.
template <int WHICH>
__global__ void loops_tc_xsum(XsArgs x)
{
    extern __shared__ float2 ptab[];   // [Lf] e^{-2 pi i n / Lf}
    const int Lf = x.Lf;
    for (int n = threadIdx.x; n < Lf; n += blockDim.x) {
        float sn, cs;
        sincospif(2.0f * (float)n / (float)Lf, &sn, &cs);
        ptab[n] = make_float2(cs, -sn);
    }
    __syncthreads();
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)x.n_groups * COLS * ROWS) return;
    const int r = (int)(idx % ROWS), j = (int)((idx / ROWS) % COLS), g = (int)(idx / ((size_t)ROWS * COLS));
    const int dyi = r / NS2, ab = r % NS2;
    const int slot = g * GRP + j / NS2, cd = j % NS2;
    if (dyi >= x.ndyh || slot >= x.n_slot) return;
    float2 acc[9];
    int ix[9], inc[9];
#pragma unroll
    for (int xi = 0; xi < 9; xi++) {
        acc[xi] = make_float2(0.f, 0.f);
        ix[xi] = 0;
        inc[xi] = xi < x.ndx ? ((x.dxs[xi] % Lf) + Lf) % Lf : 0;
    }
    const float2 *w = x.W + (size_t)g * Lf * COLS * ROWS + (size_t)j * ROWS + r;
    constexpr int UB = 8;   // columns loaded ahead (independent loads in flight)
    for (int kx0 = 0; kx0 < Lf; kx0 += UB) {
        float2 vb[UB];
#pragma unroll
        for (int u = 0; u < UB; u++) vb[u] = kx0 + u < Lf ? w[(size_t)(kx0 + u) * COLS * ROWS] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < UB; u++) {
            if (kx0 + u >= Lf) break;
            const float2 v = vb[u];
#pragma unroll
            for (int xi = 0; xi < 9; xi++) {
                if (xi >= x.ndx) break;
                float2 p = ptab[ix[xi]];
                if (WHICH == 0) p.y = -p.y;
                acc[xi].x = fmaf(p.x, v.x, fmaf(-p.y, v.y, acc[xi].x));
                acc[xi].y = fmaf(p.x, v.y, fmaf(p.y, v.x, acc[xi].y));
                ix[xi] += inc[xi];
                if (ix[xi] >= Lf) ix[xi] -= Lf;
            }
        }
    }
    int sx = 0, sy = 0;
    if (WHICH == 0) {
        const int s = x.s_list ? x.s_list[slot] : slot;
        sx = (s / x.Lq) * x.nc;
        sy = (s % x.Lq) * x.nc;
    }
    const int t1 = ab / NS, t3 = ab % NS, t2 = cd / NS, t4 = cd % NS;
    const int ra = WHICH == 0 ? t2 * NS + t1 : t1 * NS + t2;
    const int cb = WHICH == 0 ? t4 * NS + t3 : t3 * NS + t4;
#pragma unroll
    for (int xi = 0; xi < 9; xi++) {
        if (xi >= x.ndx) break;
        const int di = x.dslot[xi][dyi];
        if (di < 0) continue;
        float2 v = acc[xi];
        if (WHICH == 0) {
            // e^{-i s.Delta}: index (sx dx + sy dy) mod Lf of the table
            const float2 p = ptab[(int)(((long long)sx * x.dxs[xi] + (long long)sy * x.dys[dyi]) % Lf + Lf) % Lf];
            v = make_float2(p.x * v.x - p.y * v.y, p.x * v.y + p.y * v.x);
        }
        x.acc[((size_t)slot * x.nd + di) * NS4 + ra * NS2 + cb] = v;
    }
}

}  // namespace

bool loops_tc_supported(const tufrg_model *m)
{
    int ndyh = 0;
    for (int v : m->dys) ndyh += v >= 0;
    return m->precision == TUFRG_SPLIT32 && m->ns == NS && ndyh <= NDYM && (int)m->dxs.size() <= 9 && m->Lf <= 4096;
}

size_t loops_tc_w_bytes(const tufrg_model *m)
{
    const int n_slot = m->sym ? m->n_loop_q : m->Nq;
    const size_t n_groups = (size_t)(n_slot + GRP - 1) / GRP;
    return n_groups * m->Lf * COLS * ROWS * sizeof(float2);
}

// Loop column sums of one channel on the tensor cores, then the x phases into the accumulator slots of the
// multi-orbital path (one kx range): acc[slot][d][a][b] for the half-plane d.
cudaError_t launch_loops_tc(tufrg_model *m, int ch, float2 *acc)
{
    LtArgs a{};
    a.U = m->d_U32;
    a.ft = m->d_ft32;
    a.W = m->d_loop_w;
    a.s_list = m->sym ? m->d_loop_list : nullptr;
    a.n_slot = m->sym ? m->n_loop_q : m->Nq;
    a.n_groups = (a.n_slot + GRP - 1) / GRP;
    a.n_items = a.n_groups * m->Lf;
    a.Lq = m->Lq;
    a.nc = m->nc;
    a.Lf = m->Lf;
    a.spc = (m->Lf + KB - 1) / KB;
    int ndyh = 0;
    for (int v : m->dys)
        if (v >= 0) a.dys[ndyh++] = v;
    a.ndyh = ndyh;
    a.Tp = m->d_scal;
    a.thr_factor = 1e-2f;
    a.shell_T = m->regulator == TUFRG_REG_MOMENTUM_SHELL ? (float)m->T_reg : 0.f;
    a.err = m->d_err;
    auto kern = ch == 0 ? loops_tc_kernel<0> : loops_tc_kernel<1>;
    TUFRG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
    {
        PhaseScope ps(m, PH_LOOPS);
        kern<<<std::min(a.n_items, m->sm_count), NTHREADS, SMEM_BYTES, m->stream>>>(a);
        TUFRG_CUDA_TRY(cudaGetLastError());
    }
    XsArgs x{};
    x.W = m->d_loop_w;
    x.acc = acc;
    x.s_list = a.s_list;
    x.n_slot = a.n_slot;
    x.n_groups = a.n_groups;
    x.Lq = m->Lq;
    x.nc = m->nc;
    x.Lf = m->Lf;
    x.nd = m->nd;
    x.ndx = (int)m->dxs.size();
    x.ndyh = ndyh;
    for (int i = 0; i < ndyh; i++) x.dys[i] = a.dys[i];
    for (int i = 0; i < x.ndx; i++) {
        x.dxs[i] = m->dxs[i];
        for (int jy = 0; jy < NDYM; jy++) {
            x.dslot[i][jy] = -1;
            if (jy >= ndyh) continue;
            const int dx = x.dxs[i], dy = x.dys[jy];
            if (!(dy > 0 || dx >= 0)) continue;
            for (int d = 0; d < m->nd; d++)
                if (m->deltas[2 * d] == dx && m->deltas[2 * d + 1] == dy) x.dslot[i][jy] = d;
        }
    }
    const size_t n = (size_t)a.n_groups * COLS * ROWS;
    const size_t smem = sizeof(float2) * (size_t)m->Lf;
    auto xk = ch == 0 ? loops_tc_xsum<0> : loops_tc_xsum<1>;
    if (smem > 48 * 1024) TUFRG_CUDA_TRY(cudaFuncSetAttribute(xk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhaseScope ps(m, PH_LOOPRED);
    xk<<<(unsigned)((n + 255) / 256), 256, smem, m->stream>>>(x);
    return cudaGetLastError();
}

}  // namespace tufrg

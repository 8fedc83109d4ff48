// Tensor-core V.L.V products for the split path: dX/dT(q) = c_X A(q) L(q) A(q) (Eq. RGE_spin and the
// orbital form of Eq. rge_Dmat) on 5th-generation tensor cores (tcgen05, sm_103a).
//
// Two persistent launches per right-hand side, each over the work list (channel, momentum, 128-row tile, NB-column
// tile) of every requested channel and momentum:
//   first:   T = A L    with L[k][n] gathered from the compact loops through the bond-pair table, FP32 scratch;
//   second:  dX = c T A in FP64 (exact widening on the integer pipe).
// Complex GEMM as four real MMA streams into two tensor-memory accumulators:
//   Cr += Ar Br - Ai Bi,   Ci += Ar Bi + Ai Br     (the minus by the descriptor's negate-A bit).
// Precision: 3xTF32 - every FP32 operand x is split into hi = x with the 13 low mantissa bits cleared and lo = x - hi
// (exact), and each real product is hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory.
//
// The operands are read in FP32 straight from the matrices and split inside the kernel (no packing launches).  Warp
// roles of the 672-thread CTA (one per SM):
//   warps 0-15  producers, thread (K group kg = tid / 128, row r = tid % 128): per K stage of 16 columns each thread
//               loads 4 complex values of left-operand row r and 4 of right-operand row r for the next stage into
//               registers while it splits the current one; the left operand's four TF32 planes (Re hi, Re lo,
//               Im hi, Im lo) go to tensor memory (tcgen05.st, lane = row: warp w writes lanes 32 (w % 4) ..), the
//               right operand's to shared memory in the K-major core-matrix layout;
//   warp 16     tensor-memory allocation and the MMA issuer (one thread): 24 MMAs per stage (2 K-steps x 4 real
//               products x 3 TF32 passes), the left operand read from tensor memory;
//   warps 17-20 epilogue: tensor memory -> a shared-memory tile (then the accumulator is released to the next
//               item's MMAs) -> T (FP32) or c dX (FP64) in global memory, consecutive lanes on consecutive columns.
// Three stage buffers (mbarriers full / empty); one accumulator (mbarriers acc_full / acc_empty).  Every wait is
// bounded; on time-out the kernel raises the error flag, every role stops, the MMAs in flight are waited for
// (bounded) and the tensor memory is freed.
#include "tc_common.cuh"
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int TM = 128;             // MMA M: rows per tile
constexpr int KS = 16;              // K per stage (two MMA K-steps of 8)
constexpr int NSTAGE = 3;           // stage buffers
constexpr int NPROD = 512;          // producer threads (warps 0-15)
constexpr int MMA_WARP = 16;        // warps 17-20: epilogue
constexpr int NTHREADS = 21 * 32;
constexpr int NB_MAX = 112;         // columns per tile (complex), a multiple of 16
// tensor memory: accumulator Re at [0, NB), Im at [128, 128 + NB); left operand of stage b at 256 + 64 b, plane p at
// + 16 p (K = 16 columns)
constexpr unsigned ACC_IM = 128, A_COL0 = 256, A_STAGE_COLS = 64, A_PLANE_COLS = 16;
constexpr unsigned TMEM_COLS = 512;
static_assert(A_COL0 + NSTAGE * A_STAGE_COLS <= TMEM_COLS, "tensor memory budget");

struct Dims {
    int M;          // complex matrix order (a multiple of 4)
    int nks;        // K stages covering M
    int nb;         // complex columns per tile (multiple of 16, <= 112)
    int m_tiles;    // 128-row tiles covering M
    int n_tiles;    // nb-column tiles covering M
};

// n_tiles column tiles (0: the fewest that keep NB <= 112), NB the smallest multiple of 16 covering M with them
Dims dims_of(int M, int n_tiles)
{
    Dims d{};
    d.M = M;
    d.nks = (M + KS - 1) / KS;
    d.m_tiles = (M + TM - 1) / TM;
    d.n_tiles = std::max(n_tiles, (M + NB_MAX - 1) / NB_MAX);
    d.nb = ((M + d.n_tiles - 1) / d.n_tiles + 15) / 16 * 16;
    return d;
}

struct VlvArgs {
    const float2 *A;        // [2][Nq][M][M] projections (FP32, row-major)
    const float2 *Lc;       // [2][Nq][lper] compact loops (first product)
    const int *dij;         // [nff][nff] bond pair -> bond-difference index of the compact loops
    float2 *T;              // [2][nz][M][M] first product (written by the first launch, read by the second)
    double2 *out;           // [2][Nq][M][M] second product
    const int *qlist;       // slot z -> transfer momentum (null: the slot is the momentum)
    const double *scal;     // scal[1]: the flow-scale factor of the right-hand side
    int *err;
    Dims d;
    int nff, lper, Nq, nz;
    int ch0, nch;           // channels ch0 .. ch0 + nch - 1
    int n_items;
};

// the stage's values of one producer thread: left-operand row r at K = k0 .. k0 + 3 and right-operand row r (an
// output column) at the same K
struct Vals {
    float2 a[4], b[4];
};

// one producer thread's sources for one item: the left operand's row (A in the first product, T in the second) and
// the right operand's column (the compact loops of the momentum, or A), null when the row / column is padding
struct Src {
    const float2 *a;    // row m of the left operand
    const float2 *b;    // first product: the momentum's compact loops + (n % NS2); second: column n of A
    int nj;             // first product: n / NS2 (the column's bond index)
};

template <int PH, int NS2>
__device__ __forceinline__ Src item_src(const VlvArgs &p, int ch, int z, int mt, int nt, int r)
{
    const int M = p.d.M, m = mt * TM + r, n = nt * p.d.nb + r;
    const size_t M2 = (size_t)M * M;
    const int qs = p.qlist ? p.qlist[z] : z;
    Src s{nullptr, nullptr, 0};
    if (m < M) s.a = (PH == 0 ? p.A + ((size_t)ch * p.Nq + qs) * M2 : p.T + ((size_t)ch * p.nz + z) * M2) + (size_t)m * M;
    if (r < p.d.nb && n < M) {
        if (PH == 0) {
            s.b = p.Lc + ((size_t)ch * p.Nq + qs) * p.lper + n % NS2;
            s.nj = n / NS2;
        } else {
            s.b = p.A + ((size_t)ch * p.Nq + qs) * M2 + n;
        }
    }
    return s;
}

// K = k0 .. k0 + 3 of both operands (k0 a multiple of 4; M and NS2 are multiples of 4, so the four K values lie in
// one bond block)
template <int PH, int NS2>
__device__ __forceinline__ void load_stage(const Src &src, const int *sdij, int nff, int M, int k0, Vals &v)
{
    const bool in = k0 < M;
    if (src.a && in) {
        const float4 *q = reinterpret_cast<const float4 *>(src.a + k0);
        const float4 u0 = __ldg(q), u1 = __ldg(q + 1);
        v.a[0] = make_float2(u0.x, u0.y);
        v.a[1] = make_float2(u0.z, u0.w);
        v.a[2] = make_float2(u1.x, u1.y);
        v.a[3] = make_float2(u1.z, u1.w);
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) v.a[j] = make_float2(0.f, 0.f);
    }
    if (src.b && in) {
        if (PH == 0) {
            // L[k][n] = Lc[(d(k / NS2, n / NS2) NS2 + k % NS2) NS2 + n % NS2]
            const float2 *b = src.b + ((size_t)sdij[(k0 / NS2) * nff + src.nj] * NS2 + k0 % NS2) * NS2;
#pragma unroll
            for (int j = 0; j < 4; j++) v.b[j] = __ldg(b + j * NS2);
        } else {
            const float2 *b = src.b + (size_t)k0 * M;
#pragma unroll
            for (int j = 0; j < 4; j++) v.b[j] = __ldg(b + (size_t)j * M);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) v.b[j] = make_float2(0.f, 0.f);
    }
}

// exact FP32 -> FP64 by the two formats' bit layouts with selects only (the library's widen_f also handles
// subnormals, through a call that costs the epilogue's store loop its throughput); FP32 subnormals become signed
// zeros here (products below 1.2e-38 in magnitude)
__device__ __forceinline__ double f32_to_f64(float x)
{
    const unsigned u = __float_as_uint(x), e = (u >> 23) & 0xffu, sign = u & 0x80000000u;
    const unsigned e64 = e == 0xffu ? 0x7ffu : e + 896u;
    const unsigned hi = e == 0 ? sign : sign | (e64 << 20) | ((u & 0x7fffffu) >> 3);
    const unsigned lo = e == 0 ? 0u : u << 29;
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

template <int PH, int NS2>
__global__ void __launch_bounds__(NTHREADS, 1) vlv_tc_kernel(VlvArgs p)
{
    // dynamic shared memory: NSTAGE right-operand stages, the epilogue's FP32 tile [128][NB + 2], the bond table
    extern __shared__ __align__(1024) unsigned char smem[];
    const int NB = p.d.nb, nks = p.d.nks;
    const unsigned b_plane = (unsigned)NB * KS * 4, b_stage = 4 * b_plane;   // bytes
    const int estr = NB + 2;                                                  // tile row stride (complex)
    float2 *etile = reinterpret_cast<float2 *>(smem + NSTAGE * (size_t)b_stage);
    int *sdij = reinterpret_cast<int *>(etile + (size_t)TM * estr);
    __shared__ __align__(8) unsigned long long full[NSTAGE], empty[NSTAGE], accf, acce, done;
    __shared__ unsigned tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_base)),
                     "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < NSTAGE; b++) {
            tc::mbar_init(tc::smem_u32(&full[b]), NPROD);
            tc::mbar_init(tc::smem_u32(&empty[b]), 1);
        }
        tc::mbar_init(tc::smem_u32(&accf), 1);
        tc::mbar_init(tc::smem_u32(&acce), 128);
        tc::mbar_init(tc::smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (PH == 0)
        for (int i = tid; i < p.nff * p.nff; i += NTHREADS) sdij[i] = p.dij[i];
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tmem = tmem_base;
    const int G = (int)gridDim.x;
    const int my_items = p.n_items > (int)blockIdx.x ? (p.n_items - 1 - (int)blockIdx.x) / G + 1 : 0;
    // item -> (channel, slot, row tile, column tile); column tiles fastest so that neighbouring CTAs share rows
    auto decode = [&](int item, int &ch, int &z, int &mt, int &nt) {
        nt = item % p.d.n_tiles;
        int t = item / p.d.n_tiles;
        mt = t % p.d.m_tiles;
        t /= p.d.m_tiles;
        z = t % p.nz;
        ch = p.ch0 + t / p.nz;
    };

    if (warp < MMA_WARP) {
        // ------------------------------------------------------------------ producers
        const int r = tid & 127, kg = tid >> 7;
        const unsigned lane_base = (unsigned)((warp & 3) * 32) << 16;   // this warp's tensor-memory lanes
        const int n_stages = my_items * nks;
        const int M = p.d.M, nff = p.nff;
        int li = 0, k0 = 4 * kg;   // item (local index) and first K of this thread in the stage of the loads in flight
        int ch, z, mt, nt;
        decode((int)blockIdx.x, ch, z, mt, nt);
        Src src = item_src<PH, NS2>(p, ch, z, mt, nt, r);
        Vals cur, nxt;
        if (n_stages > 0) load_stage<PH, NS2>(src, sdij, nff, M, k0, nxt);
        for (int n = 0; n < n_stages; n++) {
            cur = nxt;
            // issue the loads of stage n + 1 (they land while this stage is split and stored)
            k0 += KS;
            if (k0 >= nks * KS) {
                k0 = 4 * kg;
                if (++li < my_items) {
                    decode((int)blockIdx.x + li * G, ch, z, mt, nt);
                    src = item_src<PH, NS2>(p, ch, z, mt, nt, r);
                }
            }
            if (n + 1 < n_stages) load_stage<PH, NS2>(src, sdij, nff, M, k0, nxt);
            const int b = n % NSTAGE;
            // the MMAs that read this stage buffer NSTAGE stages ago must be complete
            int ok = 1;
            if (lane == 0) {
                if (*(volatile int *)&abort_flag) ok = 0;
                else if (n >= NSTAGE) ok = tc::mbar_wait_or_abort(tc::smem_u32(&empty[b]), ((n / NSTAGE) - 1) & 1, &abort_flag) ? 1 : 0;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicExch(&abort_flag, 1);
                    atomicExch(p.err, 1);
                }
                break;   // the whole warp leaves (the MMA thread's waits then run out or see the flag)
            }
            tc::fence_after();
            // left operand: four planes x 4 columns of this lane's row into tensor memory
            const unsigned ca = tmem + lane_base + A_COL0 + b * A_STAGE_COLS + 4 * kg;
            float h[4], l[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                h[j] = tf32_trunc(cur.a[j].x);
                l[j] = cur.a[j].x - h[j];
            }
            tc::tmem_st4(ca + 0 * A_PLANE_COLS, h[0], h[1], h[2], h[3]);
            tc::tmem_st4(ca + 1 * A_PLANE_COLS, l[0], l[1], l[2], l[3]);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                h[j] = tf32_trunc(cur.a[j].y);
                l[j] = cur.a[j].y - h[j];
            }
            tc::tmem_st4(ca + 2 * A_PLANE_COLS, h[0], h[1], h[2], h[3]);
            tc::tmem_st4(ca + 3 * A_PLANE_COLS, l[0], l[1], l[2], l[3]);
            // right operand: row r of the stage's four planes in shared memory
            if (r < NB) {
                float *pb = reinterpret_cast<float *>(smem + (size_t)b * b_stage);
                const int o = tc::core_off(r, 4 * kg, NB);
                float4 hv, lv;
                hv = make_float4(tf32_trunc(cur.b[0].x), tf32_trunc(cur.b[1].x), tf32_trunc(cur.b[2].x), tf32_trunc(cur.b[3].x));
                lv = make_float4(cur.b[0].x - hv.x, cur.b[1].x - hv.y, cur.b[2].x - hv.z, cur.b[3].x - hv.w);
                *reinterpret_cast<float4 *>(pb + 0 * (b_plane / 4) + o) = hv;
                *reinterpret_cast<float4 *>(pb + 1 * (b_plane / 4) + o) = lv;
                hv = make_float4(tf32_trunc(cur.b[0].y), tf32_trunc(cur.b[1].y), tf32_trunc(cur.b[2].y), tf32_trunc(cur.b[3].y));
                lv = make_float4(cur.b[0].y - hv.x, cur.b[1].y - hv.y, cur.b[2].y - hv.z, cur.b[3].y - hv.w);
                *reinterpret_cast<float4 *>(pb + 2 * (b_plane / 4) + o) = hv;
                *reinterpret_cast<float4 *>(pb + 3 * (b_plane / 4) + o) = lv;
            }
            tc::tmem_wait_st();
            tc::fence_smem_async();
            tc::fence_before();
            tc::mbar_arrive(tc::smem_u32(&full[b]));
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const unsigned id = tc::idesc_tf32(TM, NB, false), idn = tc::idesc_tf32(TM, NB, true);
            const unsigned tr = tmem, ti = tmem + ACC_IM;
            bool ok = true;
            int n = 0;
            for (int it = 0; it < my_items && ok; it++) {
                // the accumulator must have been read by the epilogue of the previous item
                if (it >= 1 && !tc::mbar_wait_or_abort(tc::smem_u32(&acce), (it - 1) & 1, &abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after();
                for (int s = 0; s < nks; s++, n++) {
                    const int b = n % NSTAGE;
                    if (!tc::mbar_wait_or_abort(tc::smem_u32(&full[b]), (n / NSTAGE) & 1, &abort_flag)) { ok = false; break; }
                    tc::fence_after();
                    const unsigned sb = tc::smem_u32(smem + (size_t)b * b_stage), ta = tmem + A_COL0 + b * A_STAGE_COLS;
#pragma unroll
                    for (int kk = 0; kk < KS / 8; kk++) {
                        const unsigned bo = kk * 2 * (NB / 8) * 128;
                        const unsigned arh = ta + 0 * A_PLANE_COLS + 8 * kk, arl = ta + 1 * A_PLANE_COLS + 8 * kk;
                        const unsigned aih = ta + 2 * A_PLANE_COLS + 8 * kk, ail = ta + 3 * A_PLANE_COLS + 8 * kk;
                        const unsigned long long brh = tc::smem_desc(sb + 0 * b_plane + bo, NB), brl = tc::smem_desc(sb + 1 * b_plane + bo, NB);
                        const unsigned long long bih = tc::smem_desc(sb + 2 * b_plane + bo, NB), bil = tc::smem_desc(sb + 3 * b_plane + bo, NB);
                        const unsigned first = (s == 0 && kk == 0) ? 0u : 1u;
                        tc::mma_tf32_ta(tr, arh, brh, id, first);  tc::mma_tf32_ta(tr, arh, brl, id, 1u);  tc::mma_tf32_ta(tr, arl, brh, id, 1u);
                        tc::mma_tf32_ta(tr, aih, bih, idn, 1u);    tc::mma_tf32_ta(tr, aih, bil, idn, 1u); tc::mma_tf32_ta(tr, ail, bih, idn, 1u);
                        tc::mma_tf32_ta(ti, arh, bih, id, first);  tc::mma_tf32_ta(ti, arh, bil, id, 1u);  tc::mma_tf32_ta(ti, arl, bih, id, 1u);
                        tc::mma_tf32_ta(ti, aih, brh, id, 1u);     tc::mma_tf32_ta(ti, aih, brl, id, 1u);  tc::mma_tf32_ta(ti, ail, brh, id, 1u);
                    }
                    tc::commit(tc::smem_u32(&empty[b]));
                }
                if (ok) tc::commit(tc::smem_u32(&accf));
            }
            if (!ok) {
                atomicExch(&abort_flag, 1);
                atomicExch(p.err, 1);
            }
            tc::commit(tc::smem_u32(&done));   // completion of every MMA issued above
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ epilogue: tensor memory -> global
        const int qw = warp & 3, M = p.d.M;
        const unsigned lane_off = (unsigned)(qw * 32) << 16;
        const size_t M2 = (size_t)M * M;
        for (int it = 0; it < my_items; it++) {
            int ok = 1;
            if (lane == 0) ok = tc::mbar_wait_or_abort(tc::smem_u32(&accf), it & 1, &abort_flag) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) {
                    atomicExch(&abort_flag, 1);
                    atomicExch(p.err, 1);
                }
                break;
            }
            tc::fence_after();
            // the accumulator into this warp's rows of the shared-memory tile (lane = row, two columns per 16-byte
            // store; the row stride of NB + 2 columns keeps them free of bank conflicts), then release it to the
            // next item's MMAs
            float2 *et = etile + (size_t)(qw * 32) * estr;
            for (int c0 = 0; c0 < NB; c0 += 8) {
                unsigned vr[8], vi[8];
                tc::tmem_ld8(tmem + lane_off + (unsigned)c0, vr);
                tc::tmem_ld8(tmem + lane_off + ACC_IM + (unsigned)c0, vi);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; j += 2)
                    *reinterpret_cast<float4 *>(et + (size_t)lane * estr + c0 + j) =
                        make_float4(__uint_as_float(vr[j]), __uint_as_float(vi[j]), __uint_as_float(vr[j + 1]), __uint_as_float(vi[j + 1]));
            }
            tc::fence_before();
            tc::mbar_arrive(tc::smem_u32(&acce));
            __syncwarp();
            // coalesced rows: for each of the warp's 32 rows, consecutive lanes write consecutive columns
            int ch, z, mt, nt;
            decode((int)blockIdx.x + it * G, ch, z, mt, nt);
            const int qs = p.qlist ? p.qlist[z] : z;
            const int n0 = nt * NB, ncol = min(NB, M - n0), m0 = mt * TM + qw * 32, nrow = min(32, M - m0);
            // c_X times the flow-scale factor, applied in FP32 (the products carry FP32 accuracy)
            const float c = PH == 1 ? (float)((ch == 0 ? 1.0 : 2.0) * (p.scal ? p.scal[1] : 1.0)) : 1.f;
            // two columns per lane and store (ncol and n0 are even, rows start 16-byte aligned)
            const int npair = ncol / 2;
#pragma unroll 4
            for (int rr = 0; rr < nrow; rr++) {
                const float4 *src = reinterpret_cast<const float4 *>(et + (size_t)rr * estr);
                if (PH == 0) {
                    float4 *dst = reinterpret_cast<float4 *>(p.T + ((size_t)ch * p.nz + z) * M2 + (size_t)(m0 + rr) * M + n0);
                    for (int cp = lane; cp < npair; cp += 32) dst[cp] = src[cp];
                } else {
                    double2 *dst = p.out + ((size_t)ch * p.Nq + qs) * M2 + (size_t)(m0 + rr) * M + n0;
                    for (int cp = lane; cp < npair; cp += 32) {
                        const float4 v = src[cp];
                        dst[2 * cp] = make_double2(f32_to_f64(c * v.x), f32_to_f64(c * v.y));
                        dst[2 * cp + 1] = make_double2(f32_to_f64(c * v.z), f32_to_f64(c * v.w));
                    }
                }
            }
            __syncwarp();   // the tile rows are read before the next item's accumulator overwrites them
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

template <int PH>
cudaError_t launch_phase(tufrg_model *m, const VlvArgs &a)
{
    const size_t smem = NSTAGE * 4 * (size_t)a.d.nb * KS * 4 + sizeof(float2) * (size_t)TM * (a.d.nb + 2) +
                        sizeof(int) * (size_t)a.nff * a.nff;
    void (*k)(VlvArgs) = nullptr;
    switch (m->ns * m->ns) {
    case 4: k = vlv_tc_kernel<PH, 4>; break;
    case 16: k = vlv_tc_kernel<PH, 16>; break;
    case 36: k = vlv_tc_kernel<PH, 36>; break;
    default: return cudaErrorInvalidValue;
    }
    TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<std::min(a.n_items, m->sm_count), NTHREADS, smem, m->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

// the column-tile counts the products autotuner times: the fewest (widest tiles) and one more; the second only when it
// changes the tile width and keeps it at least 16
std::vector<int> tc_tile_candidates(const tufrg_model *m)
{
    const Dims a = dims_of(m->M, 0), b = dims_of(m->M, a.n_tiles + 1);
    std::vector<int> v{a.n_tiles};
    if (b.nb != a.nb && b.nb >= 16) v.push_back(b.n_tiles);
    return v;
}

int tc_tile_width(const tufrg_model *m) { return dims_of(m->M, m->tc_ntiles).nb; }

bool tc_supported(const tufrg_model *m)
{
    const int ns2 = m->ns * m->ns;
    return m->precision == TUFRG_SPLIT32 && m->products == TUFRG_PRODUCTS_TC && (ns2 == 4 || ns2 == 16 || ns2 == 36) &&
           m->M % 4 == 0;
}

cudaError_t launch_vlv_tc(tufrg_model *m, int channel_mask, double2 *d_out, const int *qlist, int nlist)
{
    if (!m->d_T) return cudaErrorNotReady;
    const int M = m->M, ns2 = m->ns * m->ns;
    const size_t M2 = (size_t)M * M;
    PhaseScope ps(m, PH_VLV, 2);
    for (int ch = 0; ch < 2; ch++)
        if (!((channel_mask >> ch) & 1))
            TUFRG_CUDA_TRY(cudaMemsetAsync(d_out + (size_t)ch * m->Nq * M2, 0, sizeof(double2) * m->Nq * M2, m->stream));
    if (!(channel_mask & 3)) return cudaSuccess;
    VlvArgs a{};
    a.A = m->d_A32;
    a.Lc = m->d_Lc32;
    a.dij = m->d_dij;
    a.T = reinterpret_cast<float2 *>(m->d_T);
    a.out = d_out;
    a.qlist = qlist;
    a.scal = m->d_scal;
    a.err = m->d_err;
    a.d = dims_of(M, m->tc_ntiles);
    a.nff = m->nff;
    a.lper = m->nd * ns2 * ns2;
    a.Nq = m->Nq;
    a.nz = qlist ? nlist : m->Nq;
    a.ch0 = (channel_mask & 1) ? 0 : 1;
    a.nch = (channel_mask & 3) == 3 ? 2 : 1;
    a.n_items = a.nch * a.nz * a.d.m_tiles * a.d.n_tiles;
    if (a.n_items == 0) return cudaSuccess;
    TUFRG_CUDA_TRY(launch_phase<0>(m, a));
    return launch_phase<1>(m, a);
}

}  // namespace tufrg

// Tensor-core V.L.V products for the split path: dX/dT(q) = c_X A(q) L(q) A(q) (Eq. RGE_spin and the
// orbital form of Eq. rge_Dmat) on 5th-generation tensor cores (tcgen05, sm_103a).
//
// Complex GEMM C = A B as four real MMA streams into two TMEM accumulators:
//   Cr += Ar Br - Ai Bi,   Ci += Ar Bi + Ai Br     (the minus by the descriptor's negate-A bit).
// Precision: 3xTF32 - every FP32 operand x is split into hi = tf32(x) and lo = x - hi, and each real
// product is hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory, which keeps FP32-level
// accuracy on the TF32 datapath.
//
// Operands are packed once per product by small kernels into the K-major, no-swizzle core-matrix
// layout of the MMA (8 rows x 16 bytes per core matrix), as four planes (Re hi, Re lo, Im hi, Im lo)
// per (row tile, 16-wide K stage), so that one pipeline stage of one operand is a single contiguous
// block.  The GEMM kernel (one CTA = 128 output rows x NB complex columns of one transfer momentum)
// runs a two-stage pipeline: thread 0 issues one bulk copy per operand and stage (cp.async.bulk with
// mbarrier transaction counts), thread 32 issues the 24 MMAs of a stage (2 K-steps x 4 products x 3)
// and commits them to the stage's "empty" barrier, so copies of stage s + 1 overlap the MMAs of s.
// The first product writes T = A L directly in the packed left-operand layout of the second; the
// second writes c T A in FP64.  Every wait is bounded: on time-out the kernel records an error code,
// waits (bounded) for its own MMAs and for the bulk copies it issued, frees its TMEM and returns.
#include "tc_common.cuh"
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int TC_M = 128;        // MMA M (rows per CTA)
constexpr int KS = 16;           // K per pipeline stage (two MMA K-steps of 8)
constexpr int TC_THREADS = 128;
constexpr int TMEM_COLS = 512;   // Cr at [0, NB), Ci at [256, 256 + NB)
using tc::core_off;
using tc::mbar_wait;
using tc::smem_desc;
using tc::smem_u32;
using tc::tf32_hi;

__device__ __forceinline__ unsigned idesc_tf32(int nb, bool neg_a) { return tc::idesc_tf32(TC_M, nb, neg_a); }
__device__ __forceinline__ void mma(unsigned tmem, unsigned long long da, unsigned long long db, unsigned idesc, unsigned acc)
{
    tc::mma_tf32(tmem, da, db, idesc, acc);
}

struct PackDims {
    int M;          // complex matrix order
    int nks;        // K stages (16 wide) covering M
    int nb;         // complex columns per N tile (multiple of 16, <= 256)
    int m_tiles;    // 128-row tiles covering M
    int n_tiles;    // NB-column tiles covering M
};

// left operand: rows m of X[q] (M x M, row-major), K = columns; planes (Re hi, Re lo, Im hi, Im lo)
// block (q, row tile, K stage) = 4 planes of 128 x 16 floats.  Grid (m_tiles, nks, Nq), 512 threads.
__global__ void __launch_bounds__(512) pack_left_kernel(const float2 *X, PackDims pd, const int *qlist, float *out)
{
    const int rt = blockIdx.x, ks = blockIdx.y, q = blockIdx.z;   // q: packed slot
    const int qs = qlist ? qlist[q] : q;                          // transfer momentum read
    const int r = threadIdx.x & 127, kg = threadIdx.x >> 7;
    const int m = rt * TC_M + r, k0 = ks * KS + kg * 4;
    float re[4], im[4];
    const float2 *src = X + ((size_t)qs * pd.M + m) * pd.M;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float2 v = (m < pd.M && k0 + j < pd.M) ? src[k0 + j] : make_float2(0.f, 0.f);
        re[j] = v.x;
        im[j] = v.y;
    }
    float *blk = out + (((size_t)q * pd.m_tiles + rt) * pd.nks + ks) * 4 * (TC_M * KS);
    const int o = core_off(r, kg * 4, TC_M);
    float4 h, l;
    h = make_float4(tf32_hi(re[0]), tf32_hi(re[1]), tf32_hi(re[2]), tf32_hi(re[3]));
    l = make_float4(re[0] - h.x, re[1] - h.y, re[2] - h.z, re[3] - h.w);
    *reinterpret_cast<float4 *>(blk + 0 * TC_M * KS + o) = h;
    *reinterpret_cast<float4 *>(blk + 1 * TC_M * KS + o) = l;
    h = make_float4(tf32_hi(im[0]), tf32_hi(im[1]), tf32_hi(im[2]), tf32_hi(im[3]));
    l = make_float4(im[0] - h.x, im[1] - h.y, im[2] - h.z, im[3] - h.w);
    *reinterpret_cast<float4 *>(blk + 2 * TC_M * KS + o) = h;
    *reinterpret_cast<float4 *>(blk + 3 * TC_M * KS + o) = l;
}

// right operand B[k][n] of one transfer momentum as rows n, K = k: B = Y[q] (row-major) or, when gidx is
// given, the loop matrix gathered from the compact loops, B[k][n] = Lc[q][gidx[k][n]].
// Grid (n_tiles, nks, Nq), block (nb, 4).
__global__ void pack_right_kernel(const float2 *Y, const float2 *Lc, const int *gidx, int lper, PackDims pd,
                                  const int *qlist, float *out)
{
    const int nt = blockIdx.x, ks = blockIdx.y, q = blockIdx.z;   // q: packed slot
    const int qs = qlist ? qlist[q] : q;                          // transfer momentum read
    const int nl = threadIdx.x, kg = threadIdx.y;
    const int n = nt * pd.nb + nl, k0 = ks * KS + kg * 4;
    float re[4], im[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int k = k0 + j;
        float2 v = make_float2(0.f, 0.f);
        if (n < pd.M && k < pd.M)
            v = gidx ? Lc[(size_t)qs * lper + gidx[(size_t)k * pd.M + n]] : Y[((size_t)qs * pd.M + k) * pd.M + n];
        re[j] = v.x;
        im[j] = v.y;
    }
    const int R = pd.nb;
    float *blk = out + (((size_t)q * pd.n_tiles + nt) * pd.nks + ks) * 4 * ((size_t)R * KS);
    const int o = core_off(nl, kg * 4, R);
    float4 h, l;
    h = make_float4(tf32_hi(re[0]), tf32_hi(re[1]), tf32_hi(re[2]), tf32_hi(re[3]));
    l = make_float4(re[0] - h.x, re[1] - h.y, re[2] - h.z, re[3] - h.w);
    *reinterpret_cast<float4 *>(blk + 0 * R * KS + o) = h;
    *reinterpret_cast<float4 *>(blk + 1 * R * KS + o) = l;
    h = make_float4(tf32_hi(im[0]), tf32_hi(im[1]), tf32_hi(im[2]), tf32_hi(im[3]));
    l = make_float4(im[0] - h.x, im[1] - h.y, im[2] - h.z, im[3] - h.w);
    *reinterpret_cast<float4 *>(blk + 2 * R * KS + o) = h;
    *reinterpret_cast<float4 *>(blk + 3 * R * KS + o) = l;
}

struct GemmArgs {
    const float *left;      // packed left operand [Nq][m_tiles][nks][4][128 x 16]
    const float *right;     // packed right operand [Nq][n_tiles][nks][4][nb x 16]
    float *out_left;        // first product: C written as the packed left operand of the second (or null)
    double2 *out64;         // second product: scale * C, [Nq][M][M] FP64 (or null)
    int *err;
    PackDims pd;
    double scale;
    const double *scal;     // optional device scale factor (scal[1])
    const int *qlist;       // optional: packed slot z holds transfer momentum qlist[z] (out64 index)
};

__global__ void __launch_bounds__(TC_THREADS, 1) tc_cgemm_kernel(GemmArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int NB = a.pd.nb, nks = a.pd.nks;
    const unsigned a_bytes = 4u * TC_M * KS * 4u, b_bytes = 4u * (unsigned)NB * KS * 4u;
    // stage s: [A planes | B planes]; both sizes are multiples of 1024 bytes
    unsigned char *stage[2] = {smem_raw, smem_raw + a_bytes + b_bytes};
    __shared__ __align__(8) unsigned long long full[2], empty[2], done;
    __shared__ unsigned tmem_base_sh;
    __shared__ int failed;
    __shared__ int last_issued[2];   // last stage whose copies went to buffer b (-1: none)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = blockIdx.x, rt = blockIdx.y, q = blockIdx.z;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
        last_issued[0] = last_issued[1] = -1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base_sh;

    const float *lsrc = a.left + (((size_t)q * a.pd.m_tiles + rt) * nks) * (a_bytes / 4);
    const float *rsrc = a.right + (((size_t)q * a.pd.n_tiles + nt) * nks) * (b_bytes / 4);
    if (tid == 0) {
        // producer: one bulk copy per operand and stage
        for (int s = 0; s < nks; s++) {
            const int b = s & 1;
            if (s >= 2 && !mbar_wait(smem_u32(&empty[b]), ((s >> 1) - 1) & 1)) { failed = 1; break; }
            unsigned long long st;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                         : "=l"(st) : "r"(smem_u32(&full[b])), "r"(a_bytes + b_bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(stage[b])), "l"(lsrc + (size_t)s * (a_bytes / 4)), "r"(a_bytes),
                         "r"(smem_u32(&full[b])) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(stage[b] + a_bytes)), "l"(rsrc + (size_t)s * (b_bytes / 4)), "r"(b_bytes),
                         "r"(smem_u32(&full[b])) : "memory");
            last_issued[b] = s;
        }
    } else if (tid == 32) {
        // MMA issuer: per stage, 2 K-steps x (Ar Br, -Ai Bi, Ar Bi, Ai Br) x (hi hi, hi lo, lo hi)
        const unsigned id = idesc_tf32(NB, false), idn = idesc_tf32(NB, true);
        const unsigned tr = tmem, ti = tmem + 256;
        bool ok = true;
        for (int s = 0; s < nks && ok; s++) {
            const int b = s & 1;
            if (!mbar_wait(smem_u32(&full[b]), (s >> 1) & 1)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned sa = smem_u32(stage[b]), sb = sa + a_bytes;
            const unsigned pa = TC_M * KS * 4, pb = (unsigned)NB * KS * 4;   // plane strides (bytes)
#pragma unroll
            for (int kk = 0; kk < 2; kk++) {
                const unsigned ao = kk * 2 * (TC_M / 8) * 128, bo = kk * 2 * (NB / 8) * 128;
                const unsigned long long arh = smem_desc(sa + 0 * pa + ao, TC_M), arl = smem_desc(sa + 1 * pa + ao, TC_M);
                const unsigned long long aih = smem_desc(sa + 2 * pa + ao, TC_M), ail = smem_desc(sa + 3 * pa + ao, TC_M);
                const unsigned long long brh = smem_desc(sb + 0 * pb + bo, NB), brl = smem_desc(sb + 1 * pb + bo, NB);
                const unsigned long long bih = smem_desc(sb + 2 * pb + bo, NB), bil = smem_desc(sb + 3 * pb + bo, NB);
                const unsigned first = (s == 0 && kk == 0) ? 0u : 1u;
                mma(tr, arh, brh, id, first);  mma(tr, arh, brl, id, 1u);  mma(tr, arl, brh, id, 1u);
                mma(tr, aih, bih, idn, 1u);    mma(tr, aih, bil, idn, 1u); mma(tr, ail, bih, idn, 1u);
                mma(ti, arh, bih, id, first);  mma(ti, arh, bil, id, 1u);  mma(ti, arl, bih, id, 1u);
                mma(ti, aih, brh, id, 1u);     mma(ti, aih, brl, id, 1u);  mma(ti, ail, brh, id, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&empty[b]))
                         : "memory");
        }
        if (!ok) failed = 1;
        // completion of every MMA issued above
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&done))
                     : "memory");
    }
    __syncwarp();
    const bool fin = mbar_wait(smem_u32(&done), 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (!fin || failed) {
        if (tid == 0) {
            atomicExch(a.err, 1);
            // bulk copies issued into this CTA's shared memory may still be in flight (the MMA thread gave up
            // before consuming them): wait, bounded, until the last one of each buffer has landed
            for (int b = 0; b < 2; b++)
                if (last_issued[b] >= 0) (void)mbar_wait(smem_u32(&full[b]), (last_issued[b] >> 1) & 1);
        }
    } else {
        // epilogue: lane = output row; 8 TMEM columns (8 complex outputs) per load from each accumulator
        const int r = warp * 32 + lane, row = rt * TC_M + r, M = a.pd.M;
        const double scale = a.scal ? a.scale * a.scal[1] : a.scale;
        for (int c0 = 0; c0 < NB; c0 += 8) {
            unsigned vr[8], vi[8];
            const unsigned lane_off = (unsigned)(warp * 32) << 16;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]), "=r"(vr[7])
                         : "r"(tmem + lane_off + (unsigned)c0));
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]), "=r"(vi[7])
                         : "r"(tmem + lane_off + 256u + (unsigned)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int n0 = nt * NB + c0;   // first complex output column of this group
            if (a.out64) {
                if (row < M) {
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        const int n = n0 + j;
                        if (n >= M) break;
                        a.out64[((size_t)(a.qlist ? a.qlist[q] : q) * M + row) * M + n] =
                            make_double2(scale * (double)__uint_as_float(vr[j]), scale * (double)__uint_as_float(vi[j]));
                    }
                }
            } else {
                // packed left operand of the next product: row tile rt, K = n (padding columns are zero here)
#pragma unroll
                for (int g = 0; g < 2; g++) {
                    const int k = n0 + 4 * g;
                    if (k >= a.pd.nks * KS) break;
                    float *blk = a.out_left + (((size_t)q * a.pd.m_tiles + rt) * a.pd.nks + k / KS) * 4 * (TC_M * KS);
                    const int o = core_off(r, k % KS, TC_M);
                    float re[4], im[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        re[j] = __uint_as_float(vr[4 * g + j]);
                        im[j] = __uint_as_float(vi[4 * g + j]);
                    }
                    float4 h = make_float4(tf32_hi(re[0]), tf32_hi(re[1]), tf32_hi(re[2]), tf32_hi(re[3]));
                    float4 l = make_float4(re[0] - h.x, re[1] - h.y, re[2] - h.z, re[3] - h.w);
                    *reinterpret_cast<float4 *>(blk + 0 * TC_M * KS + o) = h;
                    *reinterpret_cast<float4 *>(blk + 1 * TC_M * KS + o) = l;
                    h = make_float4(tf32_hi(im[0]), tf32_hi(im[1]), tf32_hi(im[2]), tf32_hi(im[3]));
                    l = make_float4(im[0] - h.x, im[1] - h.y, im[2] - h.z, im[3] - h.w);
                    *reinterpret_cast<float4 *>(blk + 2 * TC_M * KS + o) = h;
                    *reinterpret_cast<float4 *>(blk + 3 * TC_M * KS + o) = l;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

PackDims pack_dims(const tufrg_model *m)
{
    PackDims pd{};
    pd.M = m->M;
    pd.nks = (m->M + KS - 1) / KS;
    pd.n_tiles = (m->M + 255) / 256;
    pd.nb = ((m->M + pd.n_tiles - 1) / pd.n_tiles + 15) / 16 * 16;
    pd.m_tiles = (m->M + TC_M - 1) / TC_M;
    return pd;
}

}  // namespace

bool tc_supported(const tufrg_model *m) { return m->precision == TUFRG_SPLIT32 && m->products == TUFRG_PRODUCTS_TC; }

// bytes of the packed left and right operands of all transfer momenta
void tc_pack_bytes(const tufrg_model *m, size_t *left, size_t *right)
{
    const PackDims pd = pack_dims(m);
    *left = sizeof(float) * (size_t)m->Nq * pd.m_tiles * pd.nks * 4 * TC_M * KS;
    *right = sizeof(float) * (size_t)m->Nq * pd.n_tiles * pd.nks * 4 * (size_t)pd.nb * KS;
}

cudaError_t launch_vlv_tc(tufrg_model *m, int channel_mask, double2 *d_out, const int *qlist, int nlist)
{
    if (!m->d_tc_left[0] || !m->d_tc_right || !m->d_tc_gidx) return cudaErrorNotReady;
    const PackDims pd = pack_dims(m);
    const int M = m->M, ns2 = m->ns * m->ns;
    const size_t M2 = (size_t)M * M, lper = (size_t)m->nd * ns2 * ns2;
    const size_t smem = 2 * (4 * (size_t)TC_M * KS * 4 + 4 * (size_t)pd.nb * KS * 4);
    TUFRG_CUDA_TRY(cudaFuncSetAttribute(tc_cgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nz = qlist ? nlist : m->Nq;
    const dim3 ggrid(pd.n_tiles, pd.m_tiles, nz);
    const dim3 lgrid(pd.m_tiles, pd.nks, nz), rgrid(pd.n_tiles, pd.nks, nz), rblock(pd.nb, 4);
    PhaseScope ps(m, PH_VLV, 8);
    for (int ch = 0; ch < 2; ch++) {
        double2 *o = d_out + (size_t)ch * m->Nq * M2;
        if (!((channel_mask >> ch) & 1)) {
            TUFRG_CUDA_TRY(cudaMemsetAsync(o, 0, sizeof(double2) * m->Nq * M2, m->stream));
            continue;
        }
        const float2 *A = m->d_A32 + (size_t)ch * m->Nq * M2;
        // T = A L
        pack_left_kernel<<<lgrid, 512, 0, m->stream>>>(A, pd, qlist, m->d_tc_left[0]);
        pack_right_kernel<<<rgrid, rblock, 0, m->stream>>>(nullptr, m->d_Lc32 + ch * m->Nq * lper, m->d_tc_gidx, (int)lper,
                                                           pd, qlist, m->d_tc_right);
        GemmArgs g{};
        g.left = m->d_tc_left[0];
        g.right = m->d_tc_right;
        g.out_left = m->d_tc_left[1];
        g.out64 = nullptr;
        g.err = m->d_err;
        g.pd = pd;
        g.scale = 1.0;
        g.scal = nullptr;
        g.qlist = qlist;
        tc_cgemm_kernel<<<ggrid, TC_THREADS, smem, m->stream>>>(g);
        TUFRG_CUDA_TRY(cudaGetLastError());
        // dX = c T A
        pack_right_kernel<<<rgrid, rblock, 0, m->stream>>>(A, nullptr, nullptr, 0, pd, qlist, m->d_tc_right);
        GemmArgs h = g;
        h.left = m->d_tc_left[1];
        h.out_left = nullptr;
        h.out64 = o;
        h.scale = ch == 0 ? 1.0 : 2.0;
        h.scal = m->d_scal;
        tc_cgemm_kernel<<<ggrid, TC_THREADS, smem, m->stream>>>(h);
        TUFRG_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace tufrg

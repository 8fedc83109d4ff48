// Tensor-core V.L.V products for the split path: dX/dT(q) = c_X A(q) L(q) A(q) (Eq. RGE_spin and the
// orbital form of Eq. rge_Dmat) on 5th-generation tensor cores (tcgen05, sm_103a).
//
// Complex GEMM C = A B (M x K times K x N) as one real GEMM with interleaved real/imaginary indices:
//   A'[m][2k+r] = (Re, Im) A[m][k]           (the complex row read as floats, K' = 2K)
//   B'[2k][2n] = Re B, B'[2k+1][2n] = -Im B, B'[2k][2n+1] = Im B, B'[2k+1][2n+1] = Re B
//   C'[m][2n] = Re C, C'[m][2n+1] = Im C.
// Precision: 3xTF32 - every FP32 operand x is split into hi = tf32(x) and lo = x - hi, and
// C' = A'hi B'hi + A'hi B'lo + A'lo B'hi is accumulated in FP32 in tensor memory (TMEM), which keeps
// FP32-level accuracy on the TF32 datapath.
//
// One CTA (128 threads) owns a 128-row x NT-column output tile of one transfer momentum.  Per K slice
// of KC = 32 real columns the threads stage A'hi/lo (128 x KC) and B'^T hi/lo (NT x KC) in shared memory
// in the K-major, no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix), one elected
// thread issues the tcgen05.mma instructions (M = 128, N = NT, K = 8 each) and commits them to an
// mbarrier; everybody waits (bounded) before the slice buffers are rewritten.  The epilogue reads the
// accumulator with tcgen05.ld (one TMEM lane per output row) and writes complex outputs.
// Every wait is bounded: on time-out the kernel records an error code, waits (bounded) for its own
// MMAs, frees its TMEM and returns.
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int TC_M = 128;        // MMA M (rows per CTA)
constexpr int KC = 32;           // real K per shared-memory slice
constexpr int TC_THREADS = 128;
constexpr unsigned long long TC_WAIT_LIMIT = 1ull << 20;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_hi(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of element (row r, k) in a K-major no-swizzle tile with R rows and KC columns of 4 bytes:
// core matrix (r/8, k/4) at ((k/4) * (R/8) + r/8) * 128, row r%8 at 16 bytes, element k%4 at 4 bytes.
__device__ __forceinline__ int core_off(int r, int k, int R) { return ((k >> 2) * (R >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 3) * 4; }

__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, int R)
{
    const unsigned long long lbo = (unsigned long long)((R >> 3) * 128) >> 4;   // K-adjacent core matrices
    const unsigned long long sbo = 128ull >> 4;                                  // M/N-adjacent 8-row groups
    return (unsigned long long)((addr & 0x3FFFF) >> 4) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = nt
__device__ __forceinline__ unsigned idesc_tf32(int nt)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(nt >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    for (unsigned long long it = 0; it < TC_WAIT_LIMIT; it++) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

struct TcArgs {
    const float2 *A;        // [Nq][M][M]
    const float2 *B;        // [Nq][M][M] plain, or nullptr when the loop matrix is gathered
    const float2 *Lc;       // [Nq][nd][ns2][ns2] compact loops (gather)
    const int *dij;         // [nff][nff]
    float2 *out32;          // [Nq][M][M] (pass 1) or nullptr
    double2 *out64;         // [Nq][M][M] (pass 2) or nullptr
    int *err;               // error flag (set to 1 on a wait time-out)
    int M, nff, ns2, nd, nt, tmem_cols;
    double scale;
    const double *scal;     // optional device scale factor (scal[1])
};

__global__ void __launch_bounds__(TC_THREADS) tc_cgemm_kernel(TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int NT = a.nt;
    float *Ahi = reinterpret_cast<float *>(smem);
    float *Alo = Ahi + TC_M * KC;
    float *Bhi = Alo + TC_M * KC;
    float *Blo = Bhi + NT * KC;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned tmem_base_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = blockIdx.z;
    const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * NT;   // n0 counts real (interleaved) columns
    const int M = a.M, K2 = 2 * M;
    const size_t M2 = (size_t)M * M;
    const float *Aq = reinterpret_cast<const float *>(a.A + (size_t)q * M2);
    const double scale = a.scal ? a.scale * a.scal[1] : a.scale;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(a.tmem_cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base_sh;
    const unsigned idesc = idesc_tf32(NT);
    bool ok = true;
    int slice = 0;
    for (int k0 = 0; k0 < K2; k0 += KC, slice++) {
        // ---- stage A' (rows m0.., real columns k0..k0+KC) as hi/lo
        for (int e = tid; e < TC_M * KC; e += TC_THREADS) {
            const int r = e / KC, k = e % KC;
            const int gm = m0 + r, gk = k0 + k;
            const float x = (gm < M && gk < K2) ? Aq[(size_t)gm * K2 + gk] : 0.f;
            const float hi = tf32_hi(x);
            const int o = core_off(r, k, TC_M) >> 2;
            Ahi[o] = hi;
            Alo[o] = x - hi;
        }
        // ---- stage B'^T (NT interleaved output columns x KC real K) as hi/lo, one complex B entry -> 4 reals
        for (int e = tid; e < (NT / 2) * (KC / 2); e += TC_THREADS) {
            const int nn = e % (NT / 2), kk = e / (NT / 2);      // local complex column / complex k
            const int gn = n0 / 2 + nn, gk = k0 / 2 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gn < M && gk < M) {
                if (a.B) {
                    v = a.B[(size_t)q * M2 + (size_t)gk * M + gn];
                } else {
                    const int d = a.dij[(gk / a.ns2) * a.nff + gn / a.ns2];
                    v = a.Lc[(((size_t)q * a.nd + d) * a.ns2 + gk % a.ns2) * a.ns2 + gn % a.ns2];
                }
            }
            const float vals[4] = {v.x, -v.y, v.y, v.x};   // (2n,2k), (2n,2k+1), (2n+1,2k), (2n+1,2k+1)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int r = 2 * nn + (j >> 1), k = 2 * kk + (j & 1);
                const float hi = tf32_hi(vals[j]);
                const int o = core_off(r, k, NT) >> 2;
                Bhi[o] = hi;
                Blo[o] = vals[j] - hi;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
            for (int ks = 0; ks < KC / 8; ks++) {
                const unsigned aoff = ks * 2 * (TC_M / 8) * 128, boff = ks * 2 * (NT / 8) * 128;
                const unsigned long long dah = smem_desc(ah + aoff, TC_M), dal = smem_desc(al + aoff, TC_M);
                const unsigned long long dbh = smem_desc(bh + boff, NT), dbl = smem_desc(bl + boff, NT);
                const unsigned acc0 = (slice > 0 || ks > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem), "l"(dah),
                             "l"(dbh), "r"(idesc), "r"(acc0) : "memory");
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem), "l"(dah),
                             "l"(dbl), "r"(idesc), "r"(1u) : "memory");
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem), "l"(dal),
                             "l"(dbh), "r"(idesc), "r"(1u) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar))
                         : "memory");
        }
        // the slice buffers may be rewritten only after these MMAs have read them
        if (!mbar_wait(smem_u32(&mbar), slice & 1)) { ok = false; break; }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (tid == 0) atomicExch(a.err, 1);
        mbar_wait(smem_u32(&mbar), (slice & 1));   // give in-flight MMAs a second bounded chance before TMEM is freed
    } else {
        // ---- epilogue: lane = output row; 8 TMEM columns (4 complex outputs) per load
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < NT; c0 += 8) {
            unsigned r[8];
            const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int n = (n0 + c0) / 2 + j;
                    if (n >= M) continue;
                    const float re = __uint_as_float(r[2 * j]), im = __uint_as_float(r[2 * j + 1]);
                    const size_t o = (size_t)q * M2 + (size_t)row * M + n;
                    if (a.out64) a.out64[o] = make_double2(scale * (double)re, scale * (double)im);
                    else a.out32[o] = make_float2((float)(scale * re), (float)(scale * im));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
    }
}

}  // namespace

bool tc_supported(const tufrg_model *m) { return m->precision == TUFRG_SPLIT32 && m->products == TUFRG_PRODUCTS_TC; }

cudaError_t launch_vlv_tc(tufrg_model *m, int channel_mask, double2 *d_out)
{
    const int M = m->M, ns2 = m->ns * m->ns;
    const size_t M2 = (size_t)M * M, lper = (size_t)m->Nq * m->nd * ns2 * ns2;
    // N tiling of the 2M interleaved output columns: at most 256 per tile, multiple of 16
    const int n_tiles = (2 * M + 255) / 256;
    int nt = (2 * M + n_tiles - 1) / n_tiles;
    nt = (nt + 15) / 16 * 16;
    int cols = 32;
    while (cols < nt) cols *= 2;
    const size_t smem = sizeof(float) * (2 * TC_M * KC + 2 * (size_t)nt * KC) + 64 * 1024;   // + guard
    TUFRG_CUDA_TRY(cudaFuncSetAttribute(tc_cgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const dim3 grid((2 * M + nt - 1) / nt, (M + TC_M - 1) / TC_M, m->Nq);
    PhaseScope ps(m, PH_VLV, 4);
    for (int ch = 0; ch < 2; ch++) {
        double2 *o = d_out + (size_t)ch * m->Nq * M2;
        if (!((channel_mask >> ch) & 1)) {
            TUFRG_CUDA_TRY(cudaMemsetAsync(o, 0, sizeof(double2) * m->Nq * M2, m->stream));
            continue;
        }
        TcArgs a{};
        a.A = m->d_A32 + (size_t)ch * m->Nq * M2;
        a.B = nullptr;
        a.Lc = m->d_Lc32 + ch * lper;
        a.dij = m->d_dij;
        a.out32 = reinterpret_cast<float2 *>(m->d_T);
        a.err = m->d_err;
        a.M = M; a.nff = m->nff; a.ns2 = ns2; a.nd = m->nd; a.nt = nt; a.tmem_cols = cols;
        a.scale = 1.0;
        a.scal = nullptr;
        tc_cgemm_kernel<<<grid, TC_THREADS, smem, m->stream>>>(a);           // T = A L
        TUFRG_CUDA_TRY(cudaGetLastError());
        TcArgs b = a;
        b.A = reinterpret_cast<const float2 *>(m->d_T);
        b.B = m->d_A32 + (size_t)ch * m->Nq * M2;
        b.Lc = nullptr;
        b.out32 = nullptr;
        b.out64 = o;
        b.scale = ch == 0 ? 1.0 : 2.0;
        b.scal = m->d_scal;
        tc_cgemm_kernel<<<grid, TC_THREADS, smem, m->stream>>>(b);           // dX = c T A
        TUFRG_CUDA_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace tufrg

// Tensor-core GEMMs of the loop surrogate's network (5th-generation tensor cores, tcgen05, sm_103a).
//
//   C[M][N] = op(A)[M][K] op(B)[K][N] (+ bias[N]),  FP32 accumulation in tensor memory.
//
// Training passes multiply BF16 activations by BF16 weights: kind::f16 with BF16 operands, one MMA per K-step.
// Inference keeps the activations in FP32: kind::tf32, the activations split into a TF32 part and its FP32
// remainder (a = hi + lo exactly), the BF16 weights exact in TF32, two MMAs per K-step (hi B + lo B), which keeps
// the products at FP32 accuracy.  Operands (either orientation, any size) are first packed into the K-major,
// no-swizzle core-matrix layout of the MMA, zero-padded to whole tiles, so that one pipeline stage of one operand
// is one contiguous block: [tile][K stage][plane][rows x stage K].  The GEMM kernel (one CTA = 128 rows x NB
// columns) runs a two-stage bulk-copy pipeline (thread 0 issues the copies with mbarrier transaction counts,
// thread 32 the MMAs, committed to the stage's "empty" barrier); the epilogue reads the accumulator from tensor
// memory (lane = row) and writes C with the bias.  Every wait is bounded: on time-out the kernel raises the error
// flag, waits (bounded) for its MMAs and its copies, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "tc_common.cuh"
#include "tufrg_internal.cuh"

namespace tufrg {
namespace {

constexpr int MT = 128;         // rows per CTA (MMA M)
constexpr int NMAX = 256;       // largest N tile
constexpr int KS_BYTES = 128;   // stage K in bytes per row: 64 BF16 or 32 FP32 values (8 core matrices)

template <int KIND> struct Kind;
template <> struct Kind<0> {   // BF16 x BF16 (kind::f16)
    using T = __nv_bfloat16;
    static constexpr int ELEM = 2, KSTEP = 16, A_PLANES = 1;
};
template <> struct Kind<1> {   // (FP32 hi + lo) x BF16-in-FP32 (kind::tf32)
    using T = float;
    static constexpr int ELEM = 4, KSTEP = 8, A_PLANES = 2;
};

struct Dims {
    int M, N, K;
    int m_tiles, n_tiles, nb, nks;   // nb: columns per N tile (multiple of 16), nks: K stages
};

__device__ __forceinline__ float ldf(const float *p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// Packs op(S) (rows x K, element (r, k) = S[r * ld + k], or S[k * ld + r] when transposed) into tiles of R rows:
// dst [tile][stage][plane][R x stage K] in the core-matrix layout; planes: the value (BF16 or FP32), or for an
// FP32 split operand its TF32 part and remainder.  One thread per 16-byte chunk (8 BF16 or 4 FP32 values).
template <typename TS, typename TD, int PLANES>
__global__ void pack_kernel(const TS *S, int ld, int trans, int rows, int K, int R, int tiles, int nks, TD *dst,
                            const int *skip)
{
    if (skip && *skip) return;
    constexpr int EPC = 16 / (int)sizeof(TD);                  // elements per chunk
    constexpr int KSE = KS_BYTES / (int)sizeof(TD);            // stage K in elements
    const size_t per_stage = (size_t)R * KSE;                   // elements of one plane of one stage
    const size_t total = (size_t)tiles * nks * R * (KSE / EPC);
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int c = (int)(t % (KSE / EPC));
    const size_t rest = t / (KSE / EPC);
    const int r = (int)(rest % R);
    const int s = (int)((rest / R) % nks);
    const int tile = (int)(rest / ((size_t)R * nks));
    const int row = tile * R + r, k0 = s * KSE + c * EPC;
    float v[EPC];
#pragma unroll
    for (int j = 0; j < EPC; j++) {
        const int k = k0 + j;
        v[j] = (row < rows && k < K) ? ldf(trans ? S + (size_t)k * ld + row : S + (size_t)row * ld + k) : 0.f;
    }
    // element (r, k) of a plane: core matrix (k / EPC, r / 8) at ((k / EPC) (R / 8) + r / 8) 8 EPC, row r % 8
    const size_t off = (((size_t)(c) * (R / 8) + r / 8) * 8 + (r % 8)) * EPC;
    TD *base = dst + ((size_t)tile * nks + s) * PLANES * per_stage;
    if constexpr (sizeof(TD) == 2) {
        __align__(16) __nv_bfloat16 h[EPC];
#pragma unroll
        for (int j = 0; j < EPC; j++) h[j] = __float2bfloat16(v[j]);
        *reinterpret_cast<uint4 *>(base + off) = *reinterpret_cast<const uint4 *>(h);
    } else if constexpr (PLANES == 1) {
        *reinterpret_cast<float4 *>(base + off) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        const float4 hi = make_float4(tc::tf32_hi(v[0]), tc::tf32_hi(v[1]), tc::tf32_hi(v[2]), tc::tf32_hi(v[3]));
        *reinterpret_cast<float4 *>(base + off) = hi;
        *reinterpret_cast<float4 *>(base + per_stage + off) =
            make_float4(v[0] - hi.x, v[1] - hi.y, v[2] - hi.z, v[3] - hi.w);
    }
}

// instruction descriptor: D = F32; A, B = BF16 (kind::f16) or TF32 (kind::tf32); both K-major; M = 128, N = nb
template <int KIND> __device__ __forceinline__ unsigned idesc(int nb)
{
    const unsigned fmt = KIND == 0 ? 1u : 2u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((unsigned)(nb >> 3) << 17) | ((unsigned)(MT >> 4) << 24);
}

template <int KIND> __device__ __forceinline__ void mma(unsigned tmem, unsigned long long da, unsigned long long db,
                                                        unsigned id, unsigned acc)
{
    if (KIND == 0)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem), "l"(da), "l"(db), "r"(id),
                     "r"(acc) : "memory");
    else
        tc::mma_tf32(tmem, da, db, id, acc);
}

template <int KIND>
__global__ void __launch_bounds__(128, 1) mlp_gemm_kernel(const typename Kind<KIND>::T *PA, const typename Kind<KIND>::T *PB,
                                                          float *C, int ldc, Dims d, const float *bias, int *err,
                                                          const int *skip)
{
    if (skip && *skip) return;   // uniform over the grid
    using K_ = Kind<KIND>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const unsigned a_bytes = K_::A_PLANES * MT * KS_BYTES, b_bytes = (unsigned)d.nb * KS_BYTES;
    __shared__ __align__(8) unsigned long long full[2], empty[2], done;
    __shared__ unsigned tmem_base;
    __shared__ int failed;
    __shared__ int last_issued[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nt = blockIdx.x, mt = blockIdx.y;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_base)),
                     "r"(NMAX) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(tc::smem_u32(&full[b]), 1);
            tc::mbar_init(tc::smem_u32(&empty[b]), 1);
        }
        tc::mbar_init(tc::smem_u32(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
        last_issued[0] = last_issued[1] = -1;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tmem = tmem_base;
    auto stage = [&](int b) { return smem + (size_t)b * (a_bytes + b_bytes); };
    const unsigned char *asrc = reinterpret_cast<const unsigned char *>(PA) + (size_t)mt * d.nks * a_bytes;
    const unsigned char *bsrc = reinterpret_cast<const unsigned char *>(PB) + (size_t)nt * d.nks * b_bytes;
    if (tid == 0) {
        for (int s = 0; s < d.nks; s++) {
            const int b = s & 1;
            if (s >= 2 && !tc::mbar_wait(tc::smem_u32(&empty[b]), ((s >> 1) - 1) & 1)) { failed = 1; break; }
            unsigned long long st;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                         : "=l"(st) : "r"(tc::smem_u32(&full[b])), "r"(a_bytes + b_bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(tc::smem_u32(stage(b))), "l"(asrc + (size_t)s * a_bytes), "r"(a_bytes),
                         "r"(tc::smem_u32(&full[b])) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(tc::smem_u32(stage(b) + a_bytes)), "l"(bsrc + (size_t)s * b_bytes), "r"(b_bytes),
                         "r"(tc::smem_u32(&full[b])) : "memory");
            last_issued[b] = s;
        }
    } else if (tid == 32) {
        const unsigned id = idesc<KIND>(d.nb);
        bool ok = true;
        for (int s = 0; s < d.nks && ok; s++) {
            const int b = s & 1;
            if (!tc::mbar_wait(tc::smem_u32(&full[b]), (s >> 1) & 1)) { ok = false; break; }
            tc::fence_after();
            const unsigned sa = tc::smem_u32(stage(b)), sb = sa + a_bytes;
            constexpr int NSTEP = KS_BYTES / (K_::KSTEP * K_::ELEM);   // MMA K-steps per stage (4)
#pragma unroll
            for (int kk = 0; kk < NSTEP; kk++) {
                // one K-step spans two core matrices along K
                const unsigned ao = kk * 2 * (MT / 8) * 128, bo = kk * 2 * (d.nb / 8) * 128;
                const unsigned first = (s == 0 && kk == 0) ? 0u : 1u;
                const unsigned long long db = tc::smem_desc(sb + bo, d.nb);
                mma<KIND>(tmem, tc::smem_desc(sa + ao, MT), db, id, first);
                if (K_::A_PLANES == 2) mma<KIND>(tmem, tc::smem_desc(sa + MT * KS_BYTES + ao, MT), db, id, 1u);
            }
            tc::commit(tc::smem_u32(&empty[b]));
        }
        if (!ok) failed = 1;
        tc::commit(tc::smem_u32(&done));
    }
    __syncwarp();
    const bool fin = tc::mbar_wait(tc::smem_u32(&done), 0);
    tc::fence_after();
    __syncthreads();
    if (!fin || failed) {
        if (tid == 0) {
            atomicExch(err, 1);
            for (int b = 0; b < 2; b++)   // copies still in flight into this CTA's shared memory
                if (last_issued[b] >= 0) (void)tc::mbar_wait(tc::smem_u32(&full[b]), (last_issued[b] >> 1) & 1);
        }
    } else {
        const int row = mt * MT + warp * 32 + lane;
        const unsigned lane_off = (unsigned)(warp * 32) << 16;
        for (int c0 = 0; c0 < d.nb; c0 += 8) {
            unsigned v[8];
            tc::tmem_ld8(tmem + lane_off + (unsigned)c0, v);
            tc::tmem_wait_ld();
            if (row < d.M) {
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int col = nt * d.nb + c0 + j;
                    if (col < d.N) C[(size_t)row * ldc + col] = __uint_as_float(v[j]) + (bias ? bias[col] : 0.f);
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NMAX) : "memory");
    }
}

Dims dims(int M, int N, int K, int elem)
{
    Dims d{};
    d.M = M; d.N = N; d.K = K;
    d.m_tiles = (M + MT - 1) / MT;
    d.n_tiles = (N + NMAX - 1) / NMAX;
    d.nb = ((N + d.n_tiles - 1) / d.n_tiles + 15) / 16 * 16;
    const int kse = KS_BYTES / elem;
    d.nks = (K + kse - 1) / kse;
    return d;
}

}  // namespace

size_t mlp_tc_scratch_bytes(int M, int N, int K)
{
    // the larger of the two kinds (FP32 planes: A split in two, B one plane)
    const Dims d = dims(M, N, K, 4);
    return (size_t)(d.m_tiles * 2 * MT + d.n_tiles * d.nb) * d.nks * KS_BYTES;
}

// C = op(A) op(B) (+ bias): A BF16 (kind::f16) or FP32 (kind::tf32, split), B BF16; packed operands in ws
// (mlp_tc_scratch_bytes(M, N, K) bytes, 16-byte aligned)
template <typename TA>
cudaError_t mlp_gemm_tc(cudaStream_t s, const TA *A, int lda, int ta, const __nv_bfloat16 *B, int ldb, int tb, float *C,
                        int ldc, int M, int N, int K, const float *bias, const int *skip, void *ws, int *err)
{
    constexpr int KIND = sizeof(TA) == 2 ? 0 : 1;
    using T = typename Kind<KIND>::T;
    const Dims d = dims(M, N, K, Kind<KIND>::ELEM);
    T *pa = reinterpret_cast<T *>(ws);
    T *pb = pa + (size_t)d.m_tiles * d.nks * Kind<KIND>::A_PLANES * MT * (KS_BYTES / sizeof(T));
    constexpr int EPC = 16 / (int)sizeof(T), KSE = KS_BYTES / (int)sizeof(T);
    const size_t na = (size_t)d.m_tiles * d.nks * MT * (KSE / EPC), nbk = (size_t)d.n_tiles * d.nks * d.nb * (KSE / EPC);
    // A rows = M (K along a row unless transposed); B as rows n of op(B)^T: element (n, k) = op(B)[k][n]
    pack_kernel<TA, T, Kind<KIND>::A_PLANES><<<(unsigned)((na + 255) / 256), 256, 0, s>>>(A, lda, ta, M, K, MT, d.m_tiles,
                                                                                          d.nks, pa, skip);
    pack_kernel<__nv_bfloat16, T, 1><<<(unsigned)((nbk + 255) / 256), 256, 0, s>>>(B, ldb, !tb, N, K, d.nb, d.n_tiles,
                                                                                   d.nks, pb, skip);
    TUFRG_CUDA_TRY(cudaGetLastError());
    const size_t smem = 2 * (size_t)(Kind<KIND>::A_PLANES * MT + d.nb) * KS_BYTES;
    auto k = mlp_gemm_kernel<KIND>;
    TUFRG_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<dim3(d.n_tiles, d.m_tiles), 128, smem, s>>>(pa, pb, C, ldc, d, bias, err, skip);
    return cudaGetLastError();
}

template cudaError_t mlp_gemm_tc<__nv_bfloat16>(cudaStream_t, const __nv_bfloat16 *, int, int, const __nv_bfloat16 *, int,
                                                int, float *, int, int, int, int, const float *, const int *, void *, int *);
template cudaError_t mlp_gemm_tc<float>(cudaStream_t, const float *, int, int, const __nv_bfloat16 *, int, int, float *,
                                        int, int, int, int, const float *, const int *, void *, int *);

}  // namespace tufrg

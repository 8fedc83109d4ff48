// tcgen05 building blocks shared by the tensor-core kernels (sm_103a): shared-memory matrix descriptors of
// the K-major no-swizzle core-matrix layout, the TF32 instruction descriptor, bounded mbarrier waits and
// thin wrappers of the tcgen05 / mbarrier instructions (inline PTX).
#pragma once

#include <cuda_runtime.h>

namespace tufrg {
namespace tc {

constexpr unsigned long long WAIT_LIMIT = 1ull << 22;   // polls of one bounded mbarrier wait

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// TF32 part of an FP32 value (round to nearest, ties away); x - tf32_hi(x) is exact in FP32
__device__ __forceinline__ float tf32_hi(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// float offset of element (row r, k) in a K-major no-swizzle plane of R rows (a multiple of 8): core
// matrix (r/8, k/4) at ((k/4) * (R/8) + r/8) * 32 floats, row r%8 at 4 floats, element k%4.
__device__ __forceinline__ int core_off(int r, int k, int R) { return ((k >> 2) * (R >> 3) + (r >> 3)) * 32 + (r & 7) * 4 + (k & 3); }

// shared-memory descriptor of such a plane starting at byte address addr (16-byte aligned)
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, int R)
{
    const unsigned long long lbo = (unsigned long long)((R >> 3) * 128) >> 4;   // K-adjacent core matrices
    const unsigned long long sbo = 128ull >> 4;                                  // M/N-adjacent 8-row groups
    return (unsigned long long)((addr & 0x3FFFF) >> 4) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, M x N; bit 13 negates A
__device__ __forceinline__ unsigned idesc_tf32(int M, int N, bool neg_a)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | (neg_a ? (1u << 13) : 0u) | ((unsigned)(N >> 3) << 17) |
           ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity)
{
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

// waits for the completion of the phase of the given parity, giving up after WAIT_LIMIT polls
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity)
{
    for (unsigned long long it = 0; it < WAIT_LIMIT; it++)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// the same, also giving up as soon as *abort (shared memory, written by other threads) is set
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned bar, unsigned parity, const volatile int *abort)
{
    for (unsigned long long it = 0; it < WAIT_LIMIT; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255u) == 255u && *abort) return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

// D[tmem] (+)= A[desc] B[desc], kind::tf32, one CTA
__device__ __forceinline__ void mma_tf32(unsigned tmem, unsigned long long da, unsigned long long db, unsigned idesc,
                                         unsigned acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem), "l"(da), "l"(db), "r"(idesc),
                 "r"(acc) : "memory");
}

// D[tmem] (+)= A[tmem] B[desc], kind::tf32, one CTA: A in tensor memory (lane = row, one column per K element)
__device__ __forceinline__ void mma_tf32_ta(unsigned tmem_d, unsigned tmem_a, unsigned long long db, unsigned idesc,
                                            unsigned acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d), "r"(tmem_a), "l"(db),
                 "r"(idesc), "r"(acc) : "memory");
}

// four / two consecutive 32-bit columns of this warp's lanes (lane i of the warp writes row 32 (warp % 4) + i); addr
// holds the warp's lane base and the first column; warp-collective
__device__ __forceinline__ void tmem_st4(unsigned addr, float v0, float v1, float v2, float v3)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(__float_as_uint(v0)),
                 "r"(__float_as_uint(v1)), "r"(__float_as_uint(v2)), "r"(__float_as_uint(v3)) : "memory");
}
__device__ __forceinline__ void tmem_st2(unsigned addr, float v0, float v1)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(__float_as_uint(v0)),
                 "r"(__float_as_uint(v1)) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// the mbarrier at bar receives one arrival once every tcgen05 operation this thread issued so far is complete
__device__ __forceinline__ void commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes to shared memory made visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 8 consecutive 32-bit TMEM columns of this warp's 32 lanes (lane i of the warp gets row 32 (warp % 4) + i)
__device__ __forceinline__ void tmem_ld8(unsigned addr, unsigned (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc
}  // namespace tufrg

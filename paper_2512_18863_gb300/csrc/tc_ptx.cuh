// Inline-PTX helpers for the 5th-generation tensor cores (tcgen05) shared by
// the kernels that issue MMAs: shared-memory matrix descriptors (no swizzle,
// K-major 8 x 16-byte core matrices), the kind::f16 instruction descriptor
// (BF16 A and B, FP32 accumulator), MMA issue and commit, mbarrier polling
// and the tensor-memory load of the epilogue.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace pdrt {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major core matrices
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version
    return d;
}

// instruction descriptor: kind::f16, D = F32, A = B = BF16, both K-major
__device__ __forceinline__ uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(void *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

// MMA issue and commit executed by a whole converged warp and performed by
// its lane 0 only: the issuing loop then runs on warp-uniform descriptors,
// which measured faster than a loop inside a one-thread branch.  The commit
// comes from the lane that issued the MMAs, so it tracks them.
//
// mma3_warp: the three products of one K step of an FP32-accurate product
// split into BF16 hi + lo parts, D += Ah.Bh (or D = Ah.Bh when accumulate is
// 0), D += Ah.Bl, D += Al.Bh.  Descriptors are passed as their low words
// (start address, LBO) and one common high word (SBO, version): all four
// share SBO, and start addresses stay inside their 14-bit field, so the
// caller advances them with 32-bit adds.
__device__ __forceinline__ void mma3_warp(uint32_t tmem_d, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl,
                                          uint32_t desc_hi, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p, t, e;\n\t.reg .u32 l;\n\t.reg .b64 a0, a1, b0, b1;\n\t"
        "mov.u32 l, %%laneid;\n\tsetp.eq.u32 e, l, 0;\n\tsetp.ne.b32 p, %7, 0;\n\tsetp.ne.b32 t, 1, 0;\n\t"
        "mov.b64 a0, {%1, %5};\n\tmov.b64 a1, {%2, %5};\n\tmov.b64 b0, {%3, %5};\n\tmov.b64 b1, {%4, %5};\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a0, b0, %6, p;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a0, b1, %6, t;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b0, %6, t;\n\t}\n" ::"r"(tmem_d),
        "r"(ah), "r"(al), "r"(bh), "r"(bl), "r"(desc_hi), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit_warp(void *mbar)
{
    asm volatile(
        "{\n\t.reg .pred e;\n\t.reg .u32 l;\n\tmov.u32 l, %%laneid;\n\tsetp.eq.u32 e, l, 0;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n" ::"r"(
            smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(void *mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

}  // namespace
}  // namespace pdrt

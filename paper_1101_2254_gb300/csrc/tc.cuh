// tc.cuh -- tcgen05 helpers shared by the kernels that contract on the tensor
// cores (the DFT convolution stages and the network's implicit-GEMM
// convolutions): shared-memory operands in the canonical K-major layout without
// swizzle (8 x 8 bf16 core matrices of 128 B; consecutive along K 128 B apart,
// consecutive 8-row groups Kp * 16 B apart), the bf16 x bf16 -> f32 MMA issued
// by one thread, bounded mbarrier waits and tensor-memory loads.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace {

constexpr unsigned kWaitLimit = 1u << 24;  // bounded spin on an mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: bf16 x bf16 -> f32, both K-major, M x N
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, int acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// element offset of (row, k) in a canonical K-major plane with Kp columns
__device__ __forceinline__ int cofs(int row, int k, int Kp)
{
    return ((row >> 3) * (Kp >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done = 0;
    for (unsigned it = 0; it < kWaitLimit && !done; ++it)
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
            "selp.u32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity));
    return done != 0;
}

// 8 consecutive fp32 columns of the calling warp's lane quarter
__device__ __forceinline__ void tmem_ld8(uint32_t addr, float* v)
{
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace

// tcgen05 helpers shared by the tensor-core kernels: shared-memory matrix
// descriptors, the kind::f16 instruction descriptor, MMA issue and commit,
// the thread-sync fences, TMEM loads, and the split of an FP32 value into
// BF16 terms.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ptx.cuh"

namespace bdct {

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                 // base offset 0, relative offsets, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc(int n, bool a_mn_major)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn_major ? (1u << 15) : 0u) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// ------------------------------------------------------------ splitting
// x = t0 + t1 + t2, each term the round-to-nearest BF16 of what is left.
template <int TERMS>
__device__ __forceinline__ void split3(float x, __nv_bfloat16 (&t)[3])
{
    t[0] = __float2bfloat16_rn(x);
    if constexpr (TERMS > 1) {
        const float r1 = x - __bfloat162float(t[0]);  // exact
        t[1] = __float2bfloat16_rn(r1);
        if constexpr (TERMS > 2) {
            const float r2 = r1 - __bfloat162float(t[1]);  // exact
            t[2] = __float2bfloat16_rn(r2);
        }
    }
}

// TMEM columns for an allocation of at least `cols`: tcgen05.alloc takes a
// power of two from 32 to 512 (any other count is an illegal instruction).
__host__ __device__ constexpr int tmem_alloc_cols(int cols)
{
    int c = 32;
    while (c < cols) c *= 2;
    return c;
}

// Byte offset of element (r, k) of a K-major operand with K = kdim columns,
// in the no-swizzle canonical layout: core matrices of 8 rows x 16 bytes
// stored as 128 contiguous bytes, K-adjacent cores 128 bytes apart (the
// descriptor's leading byte offset), M/N-adjacent cores kdim/8 * 128 bytes
// apart (its stride byte offset).
__host__ __device__ __forceinline__ int kmaj_off_bytes(int r, int k, int kdim)
{
    return (((r >> 3) * (kdim >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

}  // namespace bdct

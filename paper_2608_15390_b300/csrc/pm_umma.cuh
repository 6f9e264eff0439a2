// pm_umma.cuh -- thin inline-PTX wrappers of the 5th-generation tensor core
// (tcgen05: MMA from shared-memory descriptors into tensor memory, TMEM
// allocation and loads) and of the shared-memory mbarrier that tracks MMA
// completion, for sm_100-family targets.
//
// Operand tiles use the no-swizzle canonical layout: a tile of R rows and C
// columns of 16-bit elements is stored as 8 x 8 "core matrices" (8 rows of 16
// contiguous bytes = 128 B each), core matrix (r / 8, c / 8) at byte offset
// ((r / 8) * (C / 8) + c / 8) * 128, element (r, c) at
// (r % 8) * 16 + (c % 8) * 2 inside it.  The same image serves as a K-major
// operand (rows = M or N, columns = K) and as an MN-major one (rows = K,
// columns = M or N); in both the descriptor's leading byte offset is the
// distance between core matrices adjacent along K and its stride byte offset
// the distance between core matrices adjacent along M / N.
#pragma once
#include <cstdint>

namespace pm {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, c) in a blocked tile of C columns
__host__ __device__ __forceinline__ uint32_t blk_off(int r, int c, int C)
{
    return (uint32_t)((((r >> 3) * (C >> 3) + (c >> 3)) << 7) + ((r & 7) << 4) + ((c & 7) << 1));
}

// shared-memory matrix descriptor (no swizzle; version bits 46-47 = 1)
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// K-major operand starting at K index k0 of a tile of C columns
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t tile, int C, int k0)
{
    return umma_desc(tile + (uint32_t)(k0 >> 3) * 128u, 128u, (uint32_t)C * 16u);
}
// MN-major operand starting at K index (tile row) k0 and M/N index (column) m0
__device__ __forceinline__ uint64_t desc_mnmajor(uint32_t tile, int C, int k0, int m0)
{
    return umma_desc(tile + (uint32_t)(k0 * C * 2) + (uint32_t)(m0 >> 3) * 128u, (uint32_t)C * 16u, 128u);
}

// instruction descriptor of kind::f16: BF16 A and B, FP32 D; a_mn / b_mn:
// the operand is MN-major
__host__ __device__ __forceinline__ uint32_t umma_idesc_bf16(int M, int N, int a_mn, int b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A B^T for one K = 16 slice; one thread issues
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate));
}

// the mbarrier arrives once every MMA this thread issued so far has completed
__device__ __forceinline__ void umma_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols)  // whole warp
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)  // whole warp
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w of a
// warpgroup reads lanes 32 (w % 4) .. + 31); waits for the load
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// wait for the phase of the given parity to complete; false after `limit`
// polls (the caller records the failure and stops issuing work)
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred P1;\n\tmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(ok)
            : "r"(smem_addr(mbar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

}  // namespace pm

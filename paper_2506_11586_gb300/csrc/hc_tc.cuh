// hc_tc.cuh -- 5th-generation tensor-core (tcgen05) primitives in inline PTX:
// tensor-memory allocation, shared-memory matrix descriptors for K-major
// operands in the 128-byte swizzle layout, the f16 MMA with fp32 accumulation
// in tensor memory, its commit to an mbarrier, and tensor-memory loads.
//
// Operand layout (K-major, 128-byte swizzle; the plain layout is below): a K-block holds 64 f16 values of
// each row in one 128-byte line; 8 consecutive rows form a 1024-byte atom,
// atoms follow each other every 1024 bytes (the stride byte offset), and the
// 16-byte chunk c of row r sits at chunk position c ^ (r % 8).  The swizzle is
// applied to absolute shared-memory address bits, so every atom starts on a
// 1024-byte boundary; one MMA (K = 16) reads 32 bytes of each row, and the
// next K step of the same K-block starts 32 bytes further.
#pragma once

#include <cstdint>

#include "hc_async.cuh"

namespace hc {

// shared-memory matrix descriptor: start address (bits 0-13, 16-byte units),
// leading byte offset (bits 16-29; not used by swizzled K-major operands),
// stride byte offset (bits 32-45), the fixed value 1 at bits 46-48, base offset
// 0 (atoms 1024-byte aligned), swizzle mode 2 (128 bytes) at bits 61-63
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr, uint32_t sbo_bytes)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((sbo_bytes & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// descriptor of a K-major operand without swizzle: core matrices of 8 rows x 16
// bytes, row r of a core matrix 16 r bytes in, core matrices lbo bytes apart along
// K and sbo bytes apart along M / N (layout type 0)
__device__ __forceinline__ uint64_t tc_desc_plain(uint32_t saddr, uint32_t lbo_bytes, uint32_t sbo_bytes)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo_bytes & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo_bytes & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: D fp32 (bits 4-5 = 1), A and B f16
// (bits 7-12 = 0), both K-major (bits 15-16 = 0), N / 8 at bits 17-22, M / 16 at
// bits 24-28
__host__ __device__ constexpr uint32_t tc_idesc_f16(uint32_t M, uint32_t N)
{
    return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// ---- tensor memory -------------------------------------------------------------
// executed by one whole warp; the base address is written to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ordering of tensor-core operations around thread synchronisation
__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[M x N] (+)= A[M x K=16] . B[N x K=16]^T, issued by one thread
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// one arrival on bar once every MMA this thread has issued has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 16 consecutive 32-bit columns of this thread's lane (lane = the warp's quarter
// of the 128 lanes + its lane index)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace hc

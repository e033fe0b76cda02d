// Fifth-generation tensor cores (tcgen05, sm_100 family; built for sm_103a): operand
// descriptors, tensor-memory (TMEM) allocation, the single-thread MMA issue, its completion
// through an mbarrier, and the warp-wide TMEM loads of the accumulator.
//
// Operands live in shared memory in the canonical K-major layout without swizzling: the matrix
// is tiled into "core matrices" of 8 rows x 16 bytes (8 BF16 values per row), each stored as 128
// contiguous bytes (row r at byte 16 r).  Adjacent core matrices along K are LBO bytes apart and
// adjacent groups of 8 rows SBO bytes apart.  Here every operand uses LBO = 128 and
// SBO = (K / 8) x 128, so element (r, k) of a rows x K operand sits at byte
//   (r / 8) SBO + (k / 8) 128 + (r % 8) 16 + (k % 8) 2.
// One kind::f16 MMA consumes K = 16, i.e. two core matrices along K: the next K step starts
// 256 bytes further on.
//
// The accumulator D (M = 128 rows, FP32) occupies TMEM lanes 0..127 (row m in lane m) and one
// column per output; warp w of the CTA reads lanes 32w .. 32w + 31.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "erf_tma.cuh"

namespace erfk {

// shared-memory matrix descriptor: start address, LBO and SBO in 16-byte units, the descriptor
// version bit (46) of tcgen05, base offset 0, relative LBO, no swizzle (bits 61..63 = 0)
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: D in FP32 (bits 4..5 = 1), A and B in BF16 (bits 7..9 and
// 10..12 = 1), both K-major (bits 15, 16 = 0), N / 8 in bits 17..22, M / 16 in bits 24..28
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM allocation of ncols columns (a power of two, 32..512) by one whole warp; the address is
// written to shared memory.  Every allocation is released by tc_dealloc before the CTA exits.
__device__ __forceinline__ void tc_alloc(uint32_t *smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D (+)= A B^T for one K = 16 step, issued by a single thread; accumulate = 0 overwrites D
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the mbarrier receives one arrival once every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory writes of the generic proxy become visible to the tensor-core (async) proxy
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 (16) consecutive TMEM columns of this warp's 32 lanes: thread l receives lane (taddr lane + l).
// The load and its wait form one asm statement, so no use of the registers can be scheduled
// before the data has arrived.
#define ERF_TC_R8(b) "=r"(v[b]), "=r"(v[b + 1]), "=r"(v[b + 2]), "=r"(v[b + 3]), "=r"(v[b + 4]), "=r"(v[b + 5]), \
                     "=r"(v[b + 6]), "=r"(v[b + 7])
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : ERF_TC_R8(0), ERF_TC_R8(8), ERF_TC_R8(16), ERF_TC_R8(24)
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : ERF_TC_R8(0), ERF_TC_R8(8)
        : "r"(taddr)
        : "memory");
}
#undef ERF_TC_R8

// byte offset of element (r, k) in the canonical K-major layout of an operand with K columns
__host__ __device__ constexpr uint32_t tc_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

}  // namespace erfk

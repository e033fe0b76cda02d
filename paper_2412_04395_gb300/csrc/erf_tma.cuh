// Tensor-memory-accelerator (TMA) tile loads into shared memory, tracked by an mbarrier, for the
// 3D stencil kernels (sm_90+ PTX; built for sm_103a).  One elected thread arms the barrier with
// the tile's byte count and issues cp.async.bulk.tensor; every thread waits on the barrier's
// phase with a bounded number of try_wait polls and reports a timeout instead of spinning on.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace erfk {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 3D tiled load of the box at element coordinates (x, y, z) (x innermost).  x times the element
// size must be a multiple of 16 bytes; coordinates outside the tensor read zeros.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// bounded wait: false after max_polls unsuccessful polls (each poll may suspend the thread for a
// hardware-chosen interval)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase, int max_polls) {
    for (int n = 0; n < max_polls; ++n)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
constexpr int TMA_MAX_POLLS = 1 << 20;

}  // namespace erfk

// tma.cuh -- Tensor Memory Accelerator copies into shared memory and the mbarriers they complete
// on (inline PTX), shared by the TMA-staged kernels.
//
// A 2-D tiled copy (cp.async.bulk.tensor) moves one box of a tensor map into shared memory; the
// box's innermost coordinate times the element size must be a multiple of 16 bytes, and cells
// outside the tensor are filled with zeros.  Every wait is bounded: mbar_wait gives up after
// `limit` try_wait rounds and returns false, so that a kernel can report a copy that never
// completed instead of waiting forever.
#pragma once

#include <cuda.h>

namespace segmg {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the completion of phase `parity` (at most `limit` try_wait rounds); false on
// time-out.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit) {
    const unsigned a = smem_u32(bar);
    for (long long it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 2-D tiled TMA load of the box at column x, row y (elements; x times the element size is a
// multiple of 16 bytes) into dst (128-byte aligned), completing on bar.
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int x, int y, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

}  // namespace segmg

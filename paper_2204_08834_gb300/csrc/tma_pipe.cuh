// tma_pipe.cuh - shared-memory staging by TMA tile loads that complete on mbarriers, with
// bounded waits (every wait gives up after a fixed number of polls, so no kernel can spin
// forever on a copy that never lands; the caller records the time-out and returns).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* m, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* m, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
// 3-D tiled TMA load of one box of the spectrum (coordinates x = kx, y = ky, z = k).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            unsigned long long* m) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z),
          "r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* m, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(smem_u32(m)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* m, unsigned parity, int limit = 1 << 22) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(m, parity)) return true;
    return false;
}

}  // namespace

// sbp_tma.cuh — tensor-memory-accelerator (TMA) tile loads on an mbarrier,
// with bounded waits.
//
// One elected thread arms an mbarrier with the expected byte count and issues
// cp.async.bulk.tensor copies of a 2D box of the half spectrum into shared
// memory; every thread then waits for the barrier phase.  Waits are bounded
// by a clock budget: on expiry the kernel records an error in the plan's
// device status word and the block returns, so a lost copy can never hang
// the GPU.
#pragma once

#include <cuda.h>
#include <stdint.h>

namespace sbp {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make the barrier's initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// True when the barrier phase with the given parity completed within
// `budget` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

// 2D tile load: box at element coordinates (x, y) of the tensor map into
// shared memory at dst, completing `box bytes` on the barrier.  x times the
// element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// Device-side status and debug switches shared by the TMA kernels.
struct TmaCtl {
    int* err;            // set to 1 when a bounded wait gives up
    long long budget;    // clock cycles a wait may take
    int withhold;        // test switch: arm nothing and issue no copy, so the wait runs out
};

}  // namespace sbp

// Device helpers for tile loads by the tensor memory accelerator: mbarrier
// set-up, a bounded phase wait, and a 2-D tiled bulk tensor copy into this
// CTA's shared memory.  Included by the kernels that stream tiles this way.
#pragma once
#include <cstdint>

namespace mlsd {

// about a second of SM clocks: a wait that long means the copy will not land
constexpr long long kTileWaitClocks = 1ll << 31;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init1(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mbar) : "memory");
}

// one arrival that also expects `bytes` of copies on this phase
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes)
                 : "memory");
}

// false once kTileWaitClocks have passed without the phase of this parity completing
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
        if (clock64() - t0 > kTileWaitClocks) return false;
    }
}

// box of the 2-D tensor map starting at element (x, y) into shared memory at dst,
// completing on mbar; x * element size must be a multiple of 16 bytes
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar) : "memory");
}

}  // namespace mlsd

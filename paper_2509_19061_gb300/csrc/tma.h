// tma.h -- tensor-memory-accelerator helpers (internal): host-side tensor map
// encoding through the driver entry point, device-side mbarrier and 2D bulk
// tensor copies written as inline PTX for sm_103a.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stokes {

// Encode a 2D row-major tensor map: `width` x `height` elements of
// `elem_bytes` (4 or 8), rows `pitch_bytes` apart (a multiple of 16), box of
// box_w x box_h elements (box_w * elem_bytes a multiple of 16, both <= 256).
// Out-of-range elements of a load are filled with zeros.
cudaError_t make_tmap_2d(CUtensorMap *map, const void *base, int elem_bytes, int width, int height,
                         long pitch_bytes, int box_w, int box_h);

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the initialised barrier and prior shared-memory accesses of this
// thread visible to the async (TMA) proxy
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier for at most `limit_cycles` SM clock
// cycles (one try when limit_cycles is 0, none when it is negative).
// Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit_cycles)
{
    if (limit_cycles < 0) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (clock64() - t0 < limit_cycles)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Acquire a tensor map that lives in global memory (written before the
// kernel started) for use by this thread's bulk tensor copies.
__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

// 2D tiled bulk tensor load of the box at element (x, y) into shared memory
// (128-byte aligned), completing `bar`'s transaction count.  x * element
// size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
                 : "memory");
}
#endif

} // namespace stokes

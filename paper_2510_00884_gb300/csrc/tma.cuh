// Tensor-memory-accelerator (TMA) helpers: 2D tiled bulk copies global -> shared memory
// completed on an mbarrier, with bounded waits, and the host-side tensor-map encoding
// (cuTensorMapEncodeTiled, looked up through the runtime so that no driver library is
// linked).
//
// Rules the callers keep: the tensor's base address is 16-byte aligned, its row stride a
// multiple of 16 bytes, the box's inner extent a multiple of 16 bytes, and the innermost
// coordinate of every copy a multiple of 16 bytes / element size (checked on the host).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace commet {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One try of the phase-parity wait; true once the phase with this parity has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: at most `tries` polls (each try_wait itself suspends for a while); false if
// the phase did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int tries) {
    for (int i = 0; i < tries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 2D tiled copy of the box at (x, y) (x innermost) of the tensor map into shared memory.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// Host: a 2D row-major tensor [rows][cols] of 4- or 8-byte elements with a box of
// box_rows x box_cols. Returns false when the driver entry point is unavailable or the
// encoding is refused.
bool encode_tensor_map_2d(CUtensorMap *map, const void *base, int elem_bytes, uint64_t rows, uint64_t cols,
                          uint32_t box_rows, uint32_t box_cols);

}  // namespace commet

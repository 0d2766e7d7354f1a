// Tensor-memory-accelerator (TMA) helpers for sm_103a: 2-D tiled bulk loads
// into shared memory completed on an mbarrier, with bounded waits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace nuasm {
namespace tma {

// iterations of mbarrier.try_wait before a wait gives up (each try may
// suspend the thread briefly; the bound is well above a second of waiting)
constexpr int kSpinLimit = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous (TMA) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = kSpinLimit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// one 2-D box {x, y} of `map` into shared memory at dst (128-byte aligned);
// every map here has 8-byte elements, so x must be even (16-byte rule)
__device__ __forceinline__ void load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    if (!NUASM_IN_RANGE(x & 1, 1, dbg::kTmaLoad)) return;   // the debug library skips an odd x
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// ---- bulk tensor stores (shared -> global), tracked by bulk async-groups
// Each thread that wrote the staged data runs store_fence() before the barrier
// after which one thread issues the stores; that thread waits with
// store_wait_read() before the staging area is written again and with
// store_wait_all() before the CTA exits.
__device__ __forceinline__ void store_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one 3-D box {x, y, z} of `map` from shared memory at src (128-byte aligned);
// elements outside the tensor's extent are not written
__device__ __forceinline__ void store_3d(const CUtensorMap* map, int x, int y, int z, const void* src) {
    // the debug library skips an odd x or a negative coordinate
    if (!NUASM_IN_RANGE(x & 1, 1, dbg::kTmaStore) || !NUASM_IN_RANGE(x | y | z, 1 << 30, dbg::kTmaStore)) return;
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void store_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace tma

// Host: encode a 2-D tiled tensor map over a row-major array of 8-byte
// elements (cols x rows, row pitch in elements) with boxes of box_cols x
// box_rows; out-of-bounds elements read as zero.  Returns false when the
// driver entry point is unavailable or the array breaks the TMA alignment
// rules (16-byte base and pitch).
bool encode_map_8b(CUtensorMap* map, const void* base, int cols, int rows, int pitch, int box_cols, int box_rows);

// Host: a 3-D view {cols, planes, rows} of a row-major array of 8-byte
// elements for bulk stores: element (x, y, z) is base[(z * zstep + y) * pitch
// + x] (zstep = planes: the planes interleave by row), boxes of box_cols x
// box_planes x box_rows.  Same failure rules as encode_map_8b.
bool encode_store_map_8b(CUtensorMap* map, void* base, int cols, int planes, int rows, int pitch, int box_cols,
                         int box_planes, int box_rows);

}  // namespace nuasm

// Blackwell tensor-core and tensor-memory-accelerator wrappers (inline PTX):
// tcgen05 MMA with accumulators in tensor memory, TMA tiled loads that
// complete on an mbarrier, and the shared-memory matrix descriptors both use.
//
// Layouts used (verified on the device against exact integer products):
//  * A operand, MN-major with 128-byte swizzle: 8 K-rows of 128 bytes (64
//    16-bit elements along M) form one 1024-byte atom, exactly what a TMA
//    load with CU_TENSOR_MAP_SWIZZLE_128B writes for a box whose inner
//    extent is 128 bytes.  Leading byte offset = distance between
//    consecutive 64-element M blocks, stride byte offset = distance between
//    consecutive 8-row K groups.
//  * B operand, K-major without swizzle: core matrices of 8 N-rows x 16
//    bytes (8 K elements), 128 contiguous bytes each.  Leading byte offset =
//    distance between core matrices adjacent in K, stride byte offset =
//    between core matrices adjacent in N.
//  * D (FP32) in tensor memory: row m of the M x N result in lane m, column
//    n in column n of the allocation.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "engine.cuh"

namespace wsfft {

constexpr uint32_t TC_LAYOUT_NONE = 0;
constexpr uint32_t TC_LAYOUT_SW128 = 2;

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
    d |= (uint64_t)(layout & 7) << 61;
    return d;
}

// instruction descriptor of kind::f16 with FP32 accumulation
__host__ __device__ constexpr uint32_t tc_idesc_f16(bool bf16, bool a_mn_major, bool b_mn_major, int M, int N) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((a_mn_major ? 1u : 0u) << 15) |
           ((b_mn_major ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// warp-wide: allocate `ncols` tensor-memory columns, address written to *slot
__device__ __forceinline__ void tc_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// D (+)= A * B, issued by one thread
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on `bar` once every MMA this thread issued has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
// warp-wide: lane i reads 32 consecutive columns of tensor-memory lane (taddr lane + i)
__device__ __forceinline__ void tc_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 2D tiled TMA load of the box at (x, y) into shared memory; completes on `bar`
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
// bounded wait for phase `parity` of `bar`; false once `deadline` (%globaltimer ns) passes
__device__ __forceinline__ bool mbar_wait_deadline(uint64_t *bar, uint32_t parity, uint64_t deadline) {
    if (mbar_try_wait(bar, parity)) return true;
    while (!mbar_try_wait(bar, parity))
        if (gtimer() > deadline) return false;
    return true;
}

}  // namespace wsfft

// Helpers shared by the tcgen05 kernels: shared-memory and instruction
// descriptors of kind::f16 MMAs on K-major, no-swizzle operands (8-row x
// 16-byte core matrices), the hi / lo split of an FP32 value, bounded mbarrier
// waits and bulk copies.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace zm {

constexpr unsigned long long TC_WAIT_NS = 2000000000ull;   // 2 s bound on any wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// canonical K-major, no-swizzle offset of element (row, k) of a tile with 64 k
__device__ __forceinline__ uint32_t tile_off(int row, int kgroup) {
    return (uint32_t)((row >> 3) * 1024 + kgroup * 128 + (row & 7) * 16);
}

// K-major, no swizzle: core matrices adjacent in K are LBO = 128 B apart,
// 8-row groups SBO bytes apart (1024 when a row group holds 8 core matrices).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo_bytes = 1024) {
    const uint64_t lbo = 128, sbo = sbo_bytes;
    return (uint64_t)((addr >> 4) & 0x3FFF) | (((lbo >> 4) & 0x3FFF) << 16) | (((sbo >> 4) & 0x3FFF) << 32) |
           (1ull << 46);                      // version 1, base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t instr_desc(int n, int fp16) {
    const uint32_t ab = fp16 ? 0u : 1u;       // 0 = f16, 1 = bf16
    return (1u << 4)                          // D = f32
           | (ab << 7) | (ab << 10)           // A, B types
           | ((uint32_t)(n >> 3) << 17)       // N >> 3
           | ((uint32_t)(128 >> 4) << 24);    // M = 128
}

__device__ __forceinline__ void split2(float x, int fp16, uint16_t* hi, uint16_t* lo) {
    if (fp16) {
        const __half h = __float2half_rn(x);
        *hi = __half_as_ushort(h);
        *lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        *hi = __bfloat16_as_ushort(h);
        *lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, unsigned long long t_start) {
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(bar), "r"(phase) : "memory");
        if (done) return true;
        if (global_ns() - t_start > TC_WAIT_NS) return false;
    }
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

}  // namespace zm

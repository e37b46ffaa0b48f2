// Asynchronous copies as inline PTX: per-thread cp.async (sm_80 and later).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mpr {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Per-thread 8-byte copy global -> shared, the destination given as a
// shared-window address (from smem_addr); both addresses 8-byte aligned.
// Complete for the issuing thread once it has passed cp_async_wait_all().
__device__ __forceinline__ void cp_async8_s(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace mpr

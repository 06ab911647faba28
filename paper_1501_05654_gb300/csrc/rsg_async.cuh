// Shared-memory staging helpers of the staged stencil kernels: the packed row
// entry and the cp.async copies (16 bytes, or 4/8 bytes; a source size of 0
// zero-fills the destination, which is how ghost points are staged).
#pragma once

#include <cstdint>

namespace rsg {

// Row entry packed for shared memory: start, xmin, xmax (xmin > xmax: empty).
struct SRow {
    int32_t start;
    int16_t xmin, xmax;
};

__device__ __forceinline__ void cp_async16(unsigned smem_addr, const void *gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr), "l"(gmem),
                 "r"(src_bytes)
                 : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(unsigned smem_addr, const void *gmem, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr), "l"(gmem),
                 "n"(BYTES), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace rsg

// Self-test of the bounded-wait path (no counterpart in the paper).
//
// The pipelined stencil kernels wait on mbarrier phases with a bounded
// mbarrier.try_wait loop; when the bound runs out they record status 2, let
// their copies in flight land and return, and the host reports
// RSG_ERR_TIMEOUT while the context stays usable.  k_selftest_wait runs that
// path on purpose: one warp waits on a phase that cannot complete (expected
// count 2, a single arrival), each poll suspending for at most about a
// microsecond (suspend-time hint), so `polls` sets the wait to a few
// milliseconds at most.  Nothing is copied, so nothing is left in flight.
#include "rsg_internal.h"

namespace rsg {

__global__ void k_selftest_wait(int polls, int *err) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned a = (unsigned)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(2) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
    unsigned ok = 0;
    for (int it = 0; it < polls && !ok; ++it)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(a), "r"(0u), "r"(1000u)
                     : "memory");
    if (!ok && threadIdx.x == 0) atomicExch(err, 2);
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(a) : "memory");
}

cudaError_t launch_selftest_wait(int polls, int *err, cudaStream_t st) {
    k_selftest_wait<<<1, 32, 0, st>>>(polls, err);
    return cudaGetLastError();
}

}  // namespace rsg

// Allocation-free FP64 state norms.
//
// Some callers cannot let a library call cudaMalloc: code whose device memory
// is owned by another allocator (a framework's caching allocator or a fixed
// memory pool that must account for every byte), and latency-critical loops
// where the implicit device-wide synchronisation of cudaMalloc/cudaFree would
// stall unrelated streams.  rsg_state_norms keeps its partial sums in a
// workspace the Hamiltonian allocates on first use; this variant keeps them
// in the fixed array below instead and writes the result to a device buffer
// the caller provides, so it allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "rsg_internal.h"

namespace {

constexpr int kMaxStates = 128;   // largest S accepted
constexpr int kMaxBlocks = 128;   // partial-sum rows (one per reduction block)

// Partial sums of the norm reduction: kMaxBlocks rows of kMaxStates doubles
// (128 KiB).  Every GPU that loads the library holds this array until the
// process exits.  Host code must not use the symbol as an address: the
// device address is looked up per device below.
static __device__ __align__(256) double g_norm_partials[kMaxBlocks * kMaxStates];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// Device address of g_norm_partials on the current device (looked up once
// per device, with that device current).
rsg_status partials_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rsg::set_error(RSG_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return rsg::set_error(RSG_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev] == nullptr) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_norm_partials);
        if (e != cudaSuccess || p == nullptr)
            return rsg::set_error(RSG_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                 : "no device address for the norm partials");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RSG_OK;
}

}  // namespace

extern "C" rsg_status rsg_state_norms_noalloc(rsg_ham H, const void *psi, int64_t S, int64_t ld,
                                              double *norms2_dev, void *stream) {
    if (!H || !psi || !norms2_dev) return rsg::set_error(RSG_ERR_ARG, "NULL argument");
    rsg_dtype dt;
    int64_t P;
    double h;
    rsg::ham_info(H, &dt, &P, &h);
    if (S < 1 || ld < S) return rsg::set_error(RSG_ERR_ARG, "need 1 <= S <= ld");
    // the kernels index with 32-bit ld and point offsets
    if (ld > 0x7fffffffLL || P * ld > 0x7fffffffLL) return rsg::set_error(RSG_ERR_ARG, "ld too large");
    if (S > kMaxStates)
        return rsg::set_error(RSG_ERR_UNSUPPORTED,
                              "rsg_state_norms_noalloc handles at most 128 states (fixed workspace)");
    if (dt == RSG_C64 && ld % 2) return rsg::set_error(RSG_ERR_ARG, "complex64 blocks need an even ld");
    if (((uintptr_t)psi) % 16 || ((uintptr_t)norms2_dev) % 8)
        return rsg::set_error(RSG_ERR_ARG, "misaligned pointer");
    double *partials = nullptr;
    rsg_status s = partials_address(&partials);
    if (s != RSG_OK) return s;
    int nblk = rsg::norm_blocks(P);
    if (nblk > kMaxBlocks) nblk = kMaxBlocks;
    // every block overwrites its S partial sums before they are summed, so
    // nothing in the array needs clearing between calls
    const double h3 = h * h * h;
    cudaStream_t st = (cudaStream_t)stream;
    const cudaError_t e =
        dt == RSG_C64
            ? rsg::launch_norms<float>(psi, P, (int)ld, (int)S, h3, partials, nblk, norms2_dev, st)
            : rsg::launch_norms<double>(psi, P, (int)ld, (int)S, h3, partials, nblk, norms2_dev, st);
    if (e != cudaSuccess) return rsg::set_error(RSG_ERR_CUDA, cudaGetErrorString(e));
    return RSG_OK;
}

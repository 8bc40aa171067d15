// H·v for callers that cannot allocate device memory.
//
// gbr_hv's factored path keeps two scratch vectors (X^T and its product
// with the spin-down hop lists) in the Hamiltonian handle and allocates them
// with cudaMalloc on first use.  Some callers cannot allocate at the moment
// they multiply: code that runs under a fixed memory budget handed out by a
// host framework, or real-time loops that must never reach the allocator.
// gbr_hv_static gives them the same product with the scratch in one
// file-scope device array of fixed size, so the call itself never allocates.
#include <mutex>

#include "ham.h"

namespace gbr {

// Scratch for the two vectors of the factored path.  Reserved in device
// memory of every GPU on which this library's module is loaded, until the
// process exits; with CUDA's lazy module loading the module (and so the
// array) is loaded on the device by its first use, which may be the first
// gbr_hv_static call.
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB
__device__ __align__(256) unsigned char g_hv_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static void *g_scratch_addr[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

// Device address of g_hv_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.  The
// address is cached per device: after cudaDeviceReset it is stale, so the
// entry point must not be used after a reset of the device in this process.
static int scratch_address(void **out) {
    int dev = 0;
    GBR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(GBR_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_hv_scratch);
        if (e != cudaSuccess || !p)
            return set_error(GBR_ECUDA, "cudaGetSymbolAddress(g_hv_scratch) failed: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GBR_OK;
}

}  // namespace gbr

using namespace gbr;

extern "C" int gbr_hv_static(const gbr_ham *H, const void *d_x, void *d_y, int fp, void *stream) {
    clear_error();
    if (!H) return set_error(GBR_EINVAL, "NULL handle");
    if (fp != 32 && fp != 64) return set_error(GBR_EINVAL, "fp=%d must be 32 or 64", fp);
    if (!d_x || !d_y) return set_error(GBR_EINVAL, "NULL vector");
    const size_t s = fp == 64 ? 8 : 4;
    // both scratch vectors start on 256-byte boundaries
    const size_t half = ((size_t)H->D * s + 255) & ~(size_t)255;
    if (2 * half > kStaticScratchBytes)
        return set_error(GBR_EINVAL, "sector of %lld states needs %zu scratch bytes, more than the static %zu",
                         (long long)H->D, 2 * half, kStaticScratchBytes);
    const uintptr_t xa = (uintptr_t)d_x, ya = (uintptr_t)d_y;
    if ((xa | ya) % s) return set_error(GBR_EINVAL, "vectors must be aligned to their element size");
    const uintptr_t bytes = (uintptr_t)H->D * s;
    if (xa < ya + bytes && ya < xa + bytes) return set_error(GBR_EINVAL, "x and y overlap");
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    // Every element of both scratch vectors is written before it is read
    // (transpose, then the spin-down gather), so nothing needs clearing.
    return hv_factored_with_scratch(H, d_x, d_y, fp, (cudaStream_t)stream, base, (unsigned char *)base + half);
}

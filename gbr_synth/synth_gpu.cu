// GPU twin of the seeded input generator of gbr_synth (splitmix64 in counter
// mode, Steele, Lea and Flood).  Holds no arithmetic of the ranking / H·v /
// Lanczos method: it only fills device buffers with the same draws the numpy
// generator produces, so full-size inputs need not be copied from the host.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t draw(uint64_t seed, uint64_t i) { return mix(seed ^ (i * 0x9E3779B97F4A7C15ull)); }

__global__ void k_u64(uint64_t seed, uint64_t off, int64_t n, uint64_t mask, uint64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = draw(seed, off + (uint64_t)i) & mask;
}

__global__ void k_bounded(uint64_t seed, uint64_t off, int64_t n, uint64_t bound, uint64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __umul64hi(draw(seed, off + (uint64_t)i), bound);
}

__global__ void k_uniform(uint64_t seed, uint64_t off, int64_t n, double lo, double hi, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double f = (double)(draw(seed, off + (uint64_t)i) >> 11) * 0x1.0p-53;
        out[i] = (lo == -1.0 && hi == 1.0) ? 2.0 * f - 1.0 : lo + (hi - lo) * f;
    }
}

int grid(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

}  // namespace

extern "C" int synth_u64(uint64_t seed, uint64_t off, int64_t n, uint64_t mask, uint64_t *out, void *stream) {
    if (n <= 0) return 0;
    k_u64<<<grid(n), 256, 0, (cudaStream_t)stream>>>(seed, off, n, mask, out);
    return (int)cudaGetLastError();
}

extern "C" int synth_bounded(uint64_t seed, uint64_t off, int64_t n, uint64_t bound, uint64_t *out, void *stream) {
    if (n <= 0) return 0;
    k_bounded<<<grid(n), 256, 0, (cudaStream_t)stream>>>(seed, off, n, bound, out);
    return (int)cudaGetLastError();
}

extern "C" int synth_uniform(uint64_t seed, uint64_t off, int64_t n, double lo, double hi, double *out, void *stream) {
    if (n <= 0) return 0;
    k_uniform<<<grid(n), 256, 0, (cudaStream_t)stream>>>(seed, off, n, lo, hi, out);
    return (int)cudaGetLastError();
}

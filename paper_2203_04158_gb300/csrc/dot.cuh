// Dot-product accumulators shared by the Lanczos kernels and the fused
// Lanczos epilogue of the H·v: FP64 FMA chains for FP64 vectors; for FP32
// vectors the exact product (split by an FMA) summed in two floats, which
// gives FP64-grade dots without the FP64 pipe.
#pragma once

namespace gbr {

constexpr int kRedThreads = 256;

// two-float accumulator: hi + lo, updated with the exact product of a and b
struct FF {
    float hi, lo;
};

__device__ __forceinline__ void ff_add_prod(FF &s, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);          // a*b = p + e exactly
    const float t = s.hi + p;                // TwoSum(s.hi, p)
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (p - bp);
    s.hi = t;
    s.lo += err + e;
}

template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
    FF s{0.f, 0.f};
    __device__ __forceinline__ void add(float a, float b) { ff_add_prod(s, a, b); }
    __device__ __forceinline__ double value() const { return (double)s.hi + (double)s.lo; }
};

template <int MAXT = kRedThreads>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[MAXT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xFFFFFFFFu, r, o);
    }
    return r;   // valid in thread 0
}

}  // namespace gbr

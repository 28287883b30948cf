// Device helpers shared by the library's kernels (not by the oracle).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace vne {

// ---------------------------------------------------------------------------
// Counter-based probe generator: SplitMix64 (Steele, Lea and Flood 2014).
// out(seed, c) is the (c+1)-th output of the stream started at `seed`.
// Probe entry (i, j) of an n x s block uses the counter e = j*n + i.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

constexpr uint64_t kPowerSeedXor = 0x5851F42D4C957F2Dull;

// +1 if the top bit of out(seed, e) is clear, else -1.
__device__ __forceinline__ double rademacher(uint64_t seed, uint64_t e) {
    return (splitmix_out(seed, e) >> 63) ? -1.0 : 1.0;
}

// Box-Muller from two 53-bit uniforms: u1 in (0, 1], u2 in [0, 1).
__device__ __forceinline__ double gaussian(uint64_t seed, uint64_t e) {
    const uint64_t a = splitmix_out(seed, 2ull * e);
    const uint64_t b = splitmix_out(seed, 2ull * e + 1ull);
    const double u1 = (double)((a >> 11) + 1ull) * 0x1.0p-53;
    const double u2 = (double)(b >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793238462643383279502884 * u2);
}

// The same Box-Muller draw evaluated in FP32 (for the FP32 / bf16 paths,
// whose probe block is stored in FP32 anyway): the uniforms are the same
// 53-bit values rounded to float.
__device__ __forceinline__ float gaussian_f32(uint64_t seed, uint64_t e) {
    const uint64_t a = splitmix_out(seed, 2ull * e);
    const uint64_t b = splitmix_out(seed, 2ull * e + 1ull);
    const float u1 = (float)((double)((a >> 11) + 1ull) * 0x1.0p-53);
    const float u2 = (float)((double)(b >> 11) * 0x1.0p-53);
    return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

__device__ __forceinline__ double probe_value(int kind, uint64_t seed, uint64_t e) {
    return kind == 0 ? rademacher(seed, e) : gaussian(seed, e);
}

// ---------------------------------------------------------------------------
// Device scalar block (one per call, in the workspace).
// ---------------------------------------------------------------------------
enum ScalarSlot {
    SC_U = 0,        // interval end u
    SC_LAM = 1,      // power-method estimate p1~
    SC_TRACE = 2,    // tr R
    SC_H_CHEB = 3,   // Chebyshev estimate
    SC_H_TAYLOR = 4, // Taylor estimate
    SC_FLAGS = 5,    // error bits (stored as a double-sized slot, read as uint64)
    SC_H_LEARNED = 6, // Chebyshev estimate plus the learned correction
    SC_NORM = 8,     // power method: 3*q running sums (||y||^2, x.y, x.x) per trial
    SC_COUNT = 8 + 3 * 64
};

enum Flags : unsigned long long {
    FLAG_BAD_INTERVAL = 1ull,
    FLAG_NONFINITE = 2ull,
    FLAG_TIMEOUT = 4ull,  // a bounded device-side wait gave up
};

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block in a fixed order (deterministic); result valid in thread 0.
// `sh` must hold blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) t += sh[i];
    }
    return t;
}

template <typename T> struct Math;
template <> struct Math<double> {
    static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
};
template <> struct Math<float> {
    static __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
};

}  // namespace vne

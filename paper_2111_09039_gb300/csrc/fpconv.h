// Device helpers for the element-wise kernels on n x k blocks.
//
// FP64 instructions issue at a 64th of the FP32 rate on this GPU, and the
// FP64 <-> FP32 conversion instructions are not free either, so conversions
// on the hot blocks are done on the bit patterns with integer operations.
#pragma once

#include <cuda_runtime.h>

namespace hsim {
namespace k {

// FP64 -> FP32 with the significand truncated (zeros and values outside the
// FP32 normal range take the conversion instruction)
__device__ __forceinline__ float d2f_trunc(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 1023 - 126 || e > 1023 + 127) return (float)v;
    return __int_as_float((int)((hi & 0x80000000u) | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu)));
}

// exact FP32 -> FP64 (FP32 subnormals take the conversion instruction)
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u) return (u & 0x7fffffffu) == 0u ? __longlong_as_double((long long)(u & 0x80000000u) << 32) : (double)x;
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                            ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// x 2^e by adding e to the exponent field; zeros, subnormals and results
// outside the normal range take ldexp
__device__ __forceinline__ double scale2(double x, int e) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0 || ex + e <= 0 || ex + e >= 2047) return ldexp(x, e);
    return __longlong_as_double(b + ((long long)e << 52));
}

}  // namespace k
}  // namespace hsim

// rows strided over blockIdx.y, columns over blockIdx.x * blockDim.x +
// threadIdx.x (no index division); launch with grid_rc
#define HSIM_FOR_RC(i, rows, j, cols)                                                   \
    for (int i = blockIdx.y; i < (rows); i += gridDim.y)                                \
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < (cols); j += gridDim.x * blockDim.x)

// at most 2048 row strides: each block walks many rows (launching one block
// per row of a 10^6-row block spends the time in block scheduling)
inline dim3 grid_rc(int rows, int cols, int threads = 256) {
    const int cx = (cols + threads - 1) / threads;
    const int ry = rows < 2048 ? (rows > 0 ? rows : 1) : 2048;
    return dim3((unsigned)(cx > 0 ? cx : 1), (unsigned)ry);
}

// pack2.cuh -- two-wide arithmetic for the march kernels: FP32 pairs use the packed
// f32x2 instructions of sm_100-family GPUs (one issue slot for two lanes of work); FP64 pairs
// fall back to two scalar operations.  Every op rounds to nearest like its scalar form.
#pragma once

#include <cuda_runtime.h>

namespace mmfd {

struct F2 {
    float2 v;
};
struct D2 {
    double x, y;
};

template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = F2; };
template <> struct Pair2<double> { using type = D2; };

__device__ __forceinline__ F2 mk2(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ D2 mk2(double a, double b) { return {a, b}; }
__device__ __forceinline__ F2 bc2(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ D2 bc2(double a) { return {a, a}; }
__device__ __forceinline__ float lo(F2 a) { return a.v.x; }
__device__ __forceinline__ float hi(F2 a) { return a.v.y; }
__device__ __forceinline__ double lo(D2 a) { return a.x; }
__device__ __forceinline__ double hi(D2 a) { return a.y; }

__device__ __forceinline__ F2 add2(F2 a, F2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return {__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }

__device__ __forceinline__ D2 add2(D2 a, D2 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ D2 mul2(D2 a, D2 b) { return {a.x * b.x, a.y * b.y}; }
__device__ __forceinline__ D2 fma2(D2 a, D2 b, D2 c) { return {fma(a.x, b.x, c.x), fma(a.y, b.y, c.y)}; }
__device__ __forceinline__ D2 sub2(D2 a, D2 b) { return {a.x - b.x, a.y - b.y}; }

}  // namespace mmfd

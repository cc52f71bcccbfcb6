// Two FP32 lanes processed by one packed instruction (FFMA2 / FADD2 / FMUL2 on sm_100
// and later): the per-cell arithmetic of two neighbouring cells at once.  `f2` carries the
// lane values; its operators and vfma map to the packed round-to-nearest intrinsics, so
// an expression is never contracted (a * b + c is a multiply then an add, each rounded);
// explicit vfma calls give the fused form.  The scalar overloads (V = float, or double for
// FP64 storage) are the plain operations, so code templated on V compiles to the scalar
// arithmetic unchanged.
#pragma once
#include <cuda_runtime.h>

namespace lbm {

struct __align__(8) f2 {
    float x, y;
    f2() = default;
    __device__ __forceinline__ f2(float a) : x(a), y(a) {}
    __device__ __forceinline__ f2(float a, float b) : x(a), y(b) {}
};

__device__ __forceinline__ float2 as_float2(f2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ f2 as_f2(float2 a) { return f2(a.x, a.y); }

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return as_f2(__fadd2_rn(as_float2(a), as_float2(b))); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return as_f2(__fmul2_rn(as_float2(a), as_float2(b))); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.x, -a.y); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return a + (-b); }
__device__ __forceinline__ f2 operator/(f2 a, f2 b) { return f2(a.x / b.x, a.y / b.y); }
__device__ __forceinline__ f2 &operator+=(f2 &a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2 &operator-=(f2 &a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2 &operator*=(f2 &a, f2 b) { return a = a * b; }

__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }

// Scalar type of a lane type: the type of per-launch constants (relaxation rate, weights)
// that code templated on the lane type V combines with V.
template <class V> struct ScalarOf {
    using type = V;
};
template <> struct ScalarOf<f2> {
    using type = float;
};
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c)
{
    return as_f2(__ffma2_rn(as_float2(a), as_float2(b), as_float2(c)));
}

} // namespace lbm

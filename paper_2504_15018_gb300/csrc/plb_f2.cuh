// Two FP32 lanes in one register pair, operated on with the packed FP32 instructions of
// sm_100+ (__fadd2_rn / __fmul2_rn / __ffma2_rn): one instruction updates two cells.
#pragma once
#include <cuda_runtime.h>

namespace plb {

struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ f2(float2 a) : v(a) {}
    __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ f2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ f2(double a) : v(make_float2((float)a, (float)a)) {}
    __device__ __forceinline__ f2(int a) : v(make_float2((float)a, (float)a)) {}
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.v.x, -a.v.y); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)); }
__device__ __forceinline__ f2 &operator+=(f2 &a, f2 b) { return a = a + b; }
__device__ __forceinline__ f2 &operator-=(f2 &a, f2 b) { return a = a - b; }
__device__ __forceinline__ f2 mad(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ f2 fdiv(f2 a, f2 b) { return f2(__fdividef(a.v.x, b.v.x), __fdividef(a.v.y, b.v.y)); }
__device__ __forceinline__ f2 clamp01(f2 a) {
    return f2(fminf(fmaxf(a.v.x, 0.0f), 1.0f), fminf(fmaxf(a.v.y, 0.0f), 1.0f));
}
__device__ __forceinline__ float clamp01(float a) { return fminf(fmaxf(a, 0.0f), 1.0f); }
__device__ __forceinline__ double clamp01(double a) { return fmin(fmax(a, 0.0), 1.0); }

// Scalar type of the parameters used with an arithmetic type.
template <class T> struct ScalarOf {
    using type = T;
};
template <> struct ScalarOf<f2> {
    using type = float;
};

}  // namespace plb

// f32x2.cuh -- two binary32 values carried together: the stage kernels'
// arithmetic type when one thread owns two columns of a tile (x and x + 32).
// Every operation is the correctly rounded binary32 operation on each
// component, issued as one packed two-lane instruction; with the per-point
// addressing and shared-memory instructions also shared by the two columns
// (one 16-byte access moves two values of both), a thread does the work of
// two points for roughly the instructions of one.
#pragma once

#include <cuda_runtime.h>

namespace sbli {

struct __align__(8) f32x2 {  // 8-byte aligned: one 64-bit register pair, one 8-byte access
  float x, y;
  f32x2() = default;
  __host__ __device__ constexpr f32x2(float a, float b) : x(a), y(b) {}
  __host__ __device__ explicit f32x2(double d) : x((float)d), y((float)d) {}
  __host__ __device__ explicit f32x2(int v) : x((float)v), y((float)v) {}
};

// Packed two-lane FP32 instructions (sm_100 family).  No multiply-add
// contraction happens across these calls: products that feed a sum are
// fused explicitly with fma() where the kernel writes it.
__device__ __forceinline__ float2 as_f2(f32x2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ f32x2 from_f2(float2 a) { return f32x2(a.x, a.y); }
__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) { return from_f2(__fadd2_rn(as_f2(a), as_f2(b))); }
__device__ __forceinline__ f32x2 operator-(f32x2 a) { return f32x2(-a.x, -a.y); }
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) { return from_f2(__fadd2_rn(as_f2(a), as_f2(-b))); }
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) { return from_f2(__fmul2_rn(as_f2(a), as_f2(b))); }
__device__ __forceinline__ f32x2& operator+=(f32x2& a, f32x2 b) { return a = a + b; }
__device__ __forceinline__ f32x2& operator-=(f32x2& a, f32x2 b) { return a = a - b; }
__device__ __forceinline__ f32x2& operator*=(f32x2& a, f32x2 b) { return a = a * b; }
__device__ __forceinline__ f32x2 fma(f32x2 a, f32x2 b, f32x2 c) {
  return from_f2(__ffma2_rn(as_f2(a), as_f2(b), as_f2(c)));
}

// Values per thread of an arithmetic type and access to one of them.
template <typename T>
struct Lanes {
  static constexpr int N = 1;
};
template <>
struct Lanes<f32x2> {
  static constexpr int N = 2;
};
template <typename T>
__device__ __forceinline__ T lane(T v, int) {
  return v;
}
__device__ __forceinline__ float lane(f32x2 v, int j) { return j ? v.y : v.x; }

}  // namespace sbli

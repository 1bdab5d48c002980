// dfloat.cuh -- double-float ("double-word") arithmetic: a value is the
// unevaluated sum hi + lo of two binary32 numbers with |lo| <= ulp(hi)/2,
// about 48 significant bits, evaluated entirely on the binary32 pipe.
//
// The building blocks are the classical error-free transformations
//   2Sum (Knuth), Fast2Sum (Dekker), 2Prod via FMA,
// composed as in the double-word algorithms analysed by Joldes, Muller and
// Popescu ("Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 2017):
//   add: the "sloppy" sum (2Sum of the high parts, low parts added); its
//        error is at most a few u^2 (|x| + |y|) with u = 2^-24, i.e.
//        absolute in the operands' magnitude -- the same kind of bound a
//        binary64 operation on rounded inputs has;
//   mul: the FMA product of the high parts with both cross terms folded into
//        the error term (relative error a few u^2);
//   reciprocal: one Newton step from the binary32 reciprocal.
// Every operation is written out here from those definitions.
#pragma once

#include <cuda_runtime.h>

namespace sbli {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // exact split of a binary64 value rounded to 48 bits (hi = RN(d), lo = RN(d - hi))
  __host__ __device__ explicit dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit dfloat(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

namespace dw {

// s + t = a + b exactly, any a, b (6 flops)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float ap = __fsub_rn(s, b);
  const float bp = __fsub_rn(s, ap);
  t = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
// s + t = a + b exactly when exponent(a) >= exponent(b) (3 flops)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  t = __fsub_rn(b, __fsub_rn(s, a));
}

}  // namespace dw

// Sums and products are left unnormalised (|lo| may exceed half an ulp of
// hi by a few units): the next operation's 2Sum of the high parts and its
// FMA error terms take any hi/lo split, so the renormalising Fast2Sum is
// needed only where a value leaves the double-word form (dw_normalise).
// The error bound stays a few u^2 times the operands' magnitudes.
__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  float sh, sl;
  dw::two_sum(x.hi, y.hi, sh, sl);
  return dfloat(sh, __fadd_rn(sl, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }

__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return dfloat(p, e);
}
__device__ __forceinline__ dfloat dw_normalise(dfloat x) {
  float zh, zl;
  dw::fast_two_sum(x.hi, x.lo, zh, zl);
  return dfloat(zh, zl);
}
// x * y + z.  The binary32 and binary64 overloads keep unqualified fma()
// calls in this namespace on the hardware FMA for those types.
__device__ __forceinline__ dfloat fma(dfloat x, dfloat y, dfloat z) { return x * y + z; }
__host__ __device__ __forceinline__ float fma(float x, float y, float z) { return ::fmaf(x, y, z); }
__host__ __device__ __forceinline__ double fma(double x, double y, double z) { return ::fma(x, y, z); }

__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator-=(dfloat& x, dfloat y) { return x = x - y; }
__device__ __forceinline__ dfloat& operator*=(dfloat& x, dfloat y) { return x = x * y; }

// 1 / x: t = RN(1/x.hi), residual e = 1 - x t (FMA for the high part, the low
// part subtracted), result t + t e.
__device__ __forceinline__ dfloat dw_reciprocal(dfloat xin) {
  const dfloat x = dw_normalise(xin);
  const float t = __frcp_rn(x.hi);
  float e = __fmaf_rn(-x.hi, t, 1.0f);
  e = __fmaf_rn(-x.lo, t, e);
  float zh, zl;
  dw::fast_two_sum(t, __fmul_rn(t, e), zh, zl);
  return dfloat(zh, zl);
}

}  // namespace sbli

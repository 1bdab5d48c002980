// fpconv.cuh -- binary32 <-> binary64 conversions without the FP64 pipe.
//
// GB300 executes F2F.F64.F32 / F2F.F32.F64 on its (narrow) FP64 pipe at the
// DFMA rate, about 2 per clock per SM.  The binary32-storage stage converts
// every stage value and accumulator increment, so these re-pack the IEEE bit
// patterns with integer operations instead.  Both are exact (the widening is
// exact by nature; the narrowing rounds to nearest, ties to even, as
// __double2float_rn does); operands whose result is zero, subnormal, infinite
// or NaN take the hardware conversion.
#pragma once

#include <cuda_runtime.h>

namespace sbli {

__device__ __forceinline__ double widen_f32(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = u & 0x7F800000u;
  if (e == 0u || e == 0x7F800000u) return (double)x;
  // exponent bias 127 -> 1023 (+896 at bit 20), mantissa 23 -> 52 bits
  const unsigned hi = (((u & 0x7FFFFFFFu) >> 3) + 0x38000000u) | (u & 0x80000000u);
  const unsigned lo = u << 29;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float narrow_f64(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned eb = (hi >> 20) & 0x7FFu;
  // binary32-normal results: biased exponent 897..1150
  if (eb - 897u >= 254u) return __double2float_rn(d);
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned bits = (hi & 0x80000000u) | ((eb - 896u) << 23) | mant;
  const unsigned rest = lo & 0x1FFFFFFFu;  // the 29 bits dropped
  const unsigned half = 0x10000000u;
  bits += (rest > half || (rest == half && (bits & 1u))) ? 1u : 0u;  // carry may bump the exponent
  return __uint_as_float(bits);
}

}  // namespace sbli

namespace sbli {

// Branch-free forms used in the stage kernels.  widen_f32_fast equals the
// hardware conversion except that binary32 subnormal inputs become signed
// zero; narrow_f64_fast equals __double2float_rn except that inputs of
// magnitude below 2^-126 become signed zero and NaNs become one quiet NaN.
__device__ __forceinline__ double widen_f32_fast(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = u & 0x7F800000u;
  const unsigned sign = u & 0x80000000u;
  unsigned hi = (((u & 0x7FFFFFFFu) >> 3) + 0x38000000u) | sign;
  unsigned lo = u << 29;
  hi = (e == 0u) ? sign : hi;
  lo = (e == 0u) ? 0u : lo;
  hi = (e == 0x7F800000u) ? (hi | 0x7FF00000u) : hi;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float narrow_f64_fast(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const unsigned eb = (hi >> 20) & 0x7FFu;
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned bits = sign | ((eb - 896u) << 23) | mant;
  const unsigned rest = lo & 0x1FFFFFFFu;
  bits += (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) ? 1u : 0u;
  bits = (eb < 897u) ? sign : bits;                      // zero / below the binary32 normal range
  bits = (eb > 1150u) ? (sign | 0x7F800000u) : bits;     // overflow and infinity
  bits = (eb == 0x7FFu && (((hi & 0xFFFFFu) | lo) != 0u)) ? 0x7FFFFFFFu : bits;  // NaN
  return __uint_as_float(bits);
}

// The narrowing of the binary32 stage values and of the binary32 copy of
// the state (binary32 stages with a binary64 accumulator): round to nearest,
// ties away from zero (the same error bound as ties-to-even, half a unit in
// the last place).  One funnel shift brings the 23 kept mantissa bits and the
// low 9 exponent bits together; adding 0x40000000 rebases the exponent
// (e - 896, taken modulo 2^9, lands in bits 30..23 with bit 31 clear for
// every binary32-normal result); the first dropped bit is the rounding
// increment, whose carry moves into the exponent when the mantissa
// overflows.  Results below the binary32 normal range are signed zero;
// magnitudes of 2^128 and above, infinities and NaNs give signed infinity (a
// NaN stays NaN in the binary64 accumulator and state).
__device__ __forceinline__ float narrow_f64_rna(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned t = __funnelshift_l(lo, hi, 3) + 0x40000000u + ((lo >> 28) & 1u);
  const unsigned sign = hi & 0x80000000u;
  const unsigned eb = (hi >> 20) & 0x7FFu;
  unsigned bits = t | sign;
  bits = (eb < 897u) ? sign : bits;
  bits = (eb > 1150u) ? (sign | 0x7F800000u) : bits;
  return __uint_as_float(bits);
}

// binary64 -> double-float pair: hi = RN32(v), lo = RN32(v - hi); the
// narrowings and the widening of hi are integer re-packings, the remainder one
// DADD (exact: v - hi has at most 29 significant bits).  The stage kernels
// split binary64 stage inputs this way, and the double-float path stores its
// stage fields already split this way.
__device__ __forceinline__ void split_f64(double v, float& hi, float& lo) {
  hi = narrow_f64_fast(v);
  lo = narrow_f64_fast(v - widen_f32_fast(hi));
}

}  // namespace sbli

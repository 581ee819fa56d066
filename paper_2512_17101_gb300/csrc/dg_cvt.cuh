// FP64 <-> FP32 conversions on the integer pipe.
//
// On this GPU the FP64 pipe runs at 1/64 of the FP32 rate and also executes the hardware
// FP32 <-> FP64 conversions, which the mixed-precision kernels need per node and per face node.
// These routines do the same conversions with integer operations on the IEEE-754 bit
// patterns (binary64: 1 sign, 11 exponent bits with bias 1023, 52 fraction bits; binary32:
// 1, 8 with bias 127, 23), leaving the FP64 pipe to the arithmetic that must stay FP64.
//   widen:  exact for every finite float, signed zero, infinities and NaN (NaN stays NaN);
//           float subnormals are flushed to signed zero.
//   narrow: round to nearest, ties to even, exactly as the hardware conversion whenever the
//           result is a normal float or an infinity reached by rounding; zero maps to zero;
//           inputs whose result would be subnormal, and infinities / NaN, take the hardware
//           conversion.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dg {
namespace cvt {

__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t s = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  // binary64 exponent = e - 127 + 1023; the 23 fraction bits become the top of the 52
  uint32_t hi = s | ((e + 896u) << 20) | (m >> 3), lo = m << 29;
  if (e == 0u) {  // zero (subnormals flush to zero)
    hi = s;
    lo = 0u;
  } else if (e == 255u) {  // infinity, or NaN kept quiet and non-zero
    hi = s | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u);
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float narrow(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t s = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  // normal float results: binary64 exponents 897 .. 1150 (binary32 1 .. 254)
  if (e - 897u <= 1150u - 897u) {
    const uint32_t mant = ((hi & 0xfffffu) << 3) | (lo >> 29);      // top 23 fraction bits
    const uint32_t rnd = (lo >> 28) & 1u, sticky = lo & 0x0fffffffu;  // first dropped bit, the rest
    uint32_t v = ((e - 896u) << 23) | mant;
    v += rnd & ((sticky != 0u) | (mant & 1u));  // a carry into the exponent is the correct rounding
    return __uint_as_float(s | v);
  }
  if (e == 0u) return __uint_as_float(s);  // zero and binary64 subnormals round to zero
  return __double2float_rn(x);             // subnormal results, overflow, infinities, NaN
}

// x = hi + lo with hi = narrow(x) and lo = the residual x - hi rounded to nearest: about 48
// significant bits as a float pair.  The residual is exact in binary64 and is, in units of x's
// last place, the 29 fraction bits that narrowing dropped (less 2^29 when it rounded up); it is
// formed from them with integer operations, converted to FP32 (the rounding of the residual) and
// scaled by a power of two.  Exponents outside [2^-74, 2^127) use the FP64 subtraction and the
// hardware widening.
__device__ __forceinline__ float2 split(double x) {
  const float hi = narrow(x);
  const uint32_t xh = (uint32_t)__double2hiint(x), xl = (uint32_t)__double2loint(x);
  const uint32_t e = (xh >> 20) & 0x7ffu;
  if (e - 949u > 1150u - 949u) return make_float2(hi, narrow(x - (double)hi));  // hi may be subnormal here
  const uint32_t low = xl & 0x1fffffffu;                                   // dropped fraction bits
  const uint32_t up = ((xl >> 28) & 1u) & (((xl & 0x0fffffffu) != 0u) | ((xl >> 29) & 1u));
  const int r = up ? (int)low - (1 << 29) : (int)low;                       // residual / ulp(x), exact
  const float scale = __uint_as_float((e - 1075u + 127u) << 23);          // 2^(e - 1075), a normal float
  const float lo = __int2float_rn(r) * scale;
  return make_float2(hi, (xh >> 31) ? -lo : lo);
}

}  // namespace cvt
}  // namespace dg

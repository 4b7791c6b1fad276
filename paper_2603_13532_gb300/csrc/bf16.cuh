// bfloat16 helpers of the float32 kernels: rounding, widening, and the three-plane split that
// carries a float32 (or float64) value into the bf16 tensor-core operands.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace tks {

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_float(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

// float32 -> float64 by the bits (exact): the conversion instruction runs on GB300's float64 pipe,
// about 1/64 of the integer rate.  Normal numbers and zeros take the bit path; subnormals, infinities
// and NaN the conversion.
__device__ __forceinline__ double f32_to_f64_exact(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (e != 0u && e != 0xffu)
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
  return (double)v;
}

// v ~= hi + mid + lo with each part a bfloat16 (the float32 value to about 2^-24 relative)
__device__ __forceinline__ void split3(float v, uint16_t& h0, uint16_t& h1, uint16_t& h2) {
  h0 = bf16_bits(v);
  const float r1 = v - bf16_float(h0);
  h1 = bf16_bits(r1);
  h2 = bf16_bits(r1 - bf16_float(h1));
}
// The same for a float64 value, without float64 instructions where it can (GB300's float64 pipe
// would otherwise bound the kernels that split float64 matrices): v = f + e exactly, with f = v
// rounded to float32 (nearest-even, from the float64 bits) and e = delta 2^(E - 1075) the dropped
// bits (|delta| <= 2^28, as a float32 to 2^-24 of e); then the float32 split of f with e added to
// the first remainder.  Values outside [2^-74, 2^126) take float64 arithmetic.
__device__ __forceinline__ void split3(double v, uint16_t& h0, uint16_t& h1, uint16_t& h2) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int fe = (int)((u >> 52) & 0x7ff) - 1023 + 127;   // float32 exponent field of f
  if (fe < 53 || fe > 253) {
    h0 = bf16_bits(__double2float_rn(v));
    const double r1 = v - (double)bf16_float(h0);
    h1 = bf16_bits(__double2float_rn(r1));
    const double r2 = r1 - (double)bf16_float(h1);
    h2 = bf16_bits(__double2float_rn(r2));
    return;
  }
  const unsigned long long m53 = (u & 0xfffffffffffffull) | (1ull << 52);
  const int low = (int)(m53 & 0x1fffffffull);              // the 29 bits below float32's 24
  unsigned int m24 = (unsigned int)(m53 >> 29);
  const bool up = low > 0x10000000 || (low == 0x10000000 && (m24 & 1u));
  m24 += up ? 1u : 0u;                                     // 2^24 carries into the exponent below
  const int delta = low - (up ? 0x20000000 : 0);
  const bool neg = (u >> 63) != 0;
  const float f = __uint_as_float((neg ? 0x80000000u : 0u) | ((((unsigned int)fe - 1u) << 23) + m24));
  const float e = (float)(neg ? -delta : delta) * __uint_as_float((unsigned int)(fe - 52) << 23);
  h0 = bf16_bits(f);
  const float r1 = (f - bf16_float(h0)) + e;
  h1 = bf16_bits(r1);
  h2 = bf16_bits(r1 - bf16_float(h1));
}

}  // namespace tks

// bfloat16 helpers of the float32 kernels: rounding, widening, and the three-plane split that
// carries a float32 (or float64) value into the bf16 tensor-core operands.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace tks {

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_float(uint16_t h) { return __bfloat162float(__ushort_as_bfloat16(h)); }

// v ~= hi + mid + lo with each part a bfloat16 (the float32 value to about 2^-24 relative)
__device__ __forceinline__ void split3(float v, uint16_t& h0, uint16_t& h1, uint16_t& h2) {
  h0 = bf16_bits(v);
  const float r1 = v - bf16_float(h0);
  h1 = bf16_bits(r1);
  h2 = bf16_bits(r1 - bf16_float(h1));
}
__device__ __forceinline__ void split3(double v, uint16_t& h0, uint16_t& h1, uint16_t& h2) {
  h0 = bf16_bits(__double2float_rn(v));
  const double r1 = v - (double)bf16_float(h0);
  h1 = bf16_bits(__double2float_rn(r1));
  const double r2 = r1 - (double)bf16_float(h1);
  h2 = bf16_bits(__double2float_rn(r2));
}

}  // namespace tks

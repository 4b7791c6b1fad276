// Quotients of small non-negative integers without an integer division (about 20 instructions
// each on the CUDA cores): floor(e / d) = trunc((e + 1/2) * RN(1/d)) in float32 for 0 <= e < 2^16 and
// 1 <= d <= 256, and for 0 <= e < 2^15 and 1 <= d <= 1024.  (e + 1/2) / d lies at least 1/(2d) from an integer and the two float32 roundings
// stay inside that margin over the whole range (checked exhaustively by the CPU test suite).  The
// reciprocal is an IEEE division (the library is built without fast-math), i.e. RN(1/d).
#pragma once

namespace tks {

struct SmallDiv {
  int d;
  float rd;
  __device__ __forceinline__ explicit SmallDiv(int divisor) : d(divisor), rd(1.0f / (float)divisor) {}
  __device__ __forceinline__ int quo(int e) const { return __float2int_rz(((float)e + 0.5f) * rd); }
};

}  // namespace tks

// Counter-based Gaussian draws for the sketch matrices Omega_j (device side).
//
// The paper asks for standard Gaussian Omega_j (Sec. 3.1) reused across the sketches of
// all other modes.  Definition used here (and restated independently by the CPU oracle):
//   Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key (seed, 0) and counter
//   (block, mode, problem, stream); each 64-bit word w gives u = (floor(w/2^12) + 1/2) 2^-52;
//   Box-Muller z = sqrt(-2 ln u1) (cos, sin)(2 pi u2); lanes 0..3 of a block are
//   r(w0)cos(w1), r(w0)sin(w1), r(w2)cos(w3), r(w2)sin(w3).
// ln and (cos, sin)(2 pi u) are evaluated from textbook series (atanh series of ln after
// reduction to [sqrt(1/2), sqrt(2)); Taylor series of sin/cos on [0, pi/4] after octant
// reduction) with only correctly rounded IEEE operations in one fixed order, written with
// explicit __d*_rn intrinsics so the compiler cannot contract them into fused multiply-adds.
// Any transcription performing the same operations in the same order produces the same bits.
//
// The low-precision sketch draws in float32 instead (gaussian4_f32): the same Philox words,
// u = (floor(w/2^41) + 1/2) 2^-23 (exact in float32), the same two series with float32
// coefficients and fewer terms (5 for ln, 4 for sin, 5 for cos), explicit __f*_rn operations,
// then round-to-nearest-even to bfloat16.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace tks {
namespace rng {

constexpr uint64_t kM0 = 0xD2E7470EE14C6C93ull;  // Philox4x64 multipliers
constexpr uint64_t kM1 = 0xCA5A826395121157ull;
constexpr uint64_t kW0 = 0x9E3779B97F4A7C15ull;  // Weyl key increments
constexpr uint64_t kW1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(kM0, c[0]), lo0 = kM0 * c[0];
    const uint64_t hi1 = __umul64hi(kM1, c[2]), lo1 = kM1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0;
    const uint64_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += kW0;
    k1 += kW1;
  }
}

__device__ __forceinline__ double uniform_open01(uint64_t w) {
  return __dmul_rn(__dadd_rn(static_cast<double>(w >> 12), 0.5), 0x1p-52);
}

// ln u for u in (0, 1): u = m 2^e, m in [sqrt(1/2), sqrt(2)), f = (m-1)/(m+1), s = f^2,
// ln m = 2f + (2f s) q(s), q(s) = sum_{k>=1} s^(k-1)/(2k+1) (11 terms, Horner),
// ln u = e ln2_hi + (e ln2_lo + ln m).
__device__ __forceinline__ double ln_open01(double u) {
  const long long bits = __double_as_longlong(u);
  int e = static_cast<int>((bits >> 52) & 0x7ff) - 1022;
  double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3fe0000000000000LL);
  if (m < 0x1.6a09e667f3bcdp-1) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double f = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double s = __dmul_rn(f, f);
  // 1/(2k+1), k = 1..11, correctly rounded
  const double c[11] = {0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3,
                        0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4,
                        0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5, 0x1.af286bca1af28p-5,
                        0x1.8618618618618p-5, 0x1.642c8590b2164p-5};
  double q = c[10];
#pragma unroll
  for (int k = 9; k >= 0; --k) q = __dadd_rn(__dmul_rn(q, s), c[k]);
  const double two_f = __dmul_rn(f, 2.0);
  const double ln_m = __dadd_rn(two_f, __dmul_rn(__dmul_rn(two_f, s), q));
  const double ed = static_cast<double>(e);
  const double ln2_hi = 0x1.62e42fee00000p-1, ln2_lo = 0x1.a39ef35793c76p-33;
  return __dadd_rn(__dmul_rn(ed, ln2_hi), __dadd_rn(__dmul_rn(ed, ln2_lo), ln_m));
}

// (cos 2 pi u, sin 2 pi u) for u in (0, 1): x = 8u, k = floor x, f = x - k (both exact),
// t = (pi/4) g with g = f (k even) or 1 - f (k odd); Taylor series on [0, pi/4].
__device__ __forceinline__ void sincos_2pi(double u, double* cs, double* sn) {
  const double x = __dmul_rn(u, 8.0);
  const double kf = floor(x);
  const double f = __dsub_rn(x, kf);
  const int k = static_cast<int>(kf);
  const double g = (k & 1) ? __dsub_rn(1.0, f) : f;
  const double t = __dmul_rn(g, 0x1.921fb54442d18p-1);
  const double s2 = __dmul_rn(t, t);
  // (-1)^k/(2k+1)!, k = 1..8 and (-1)^k/(2k)!, k = 1..9, correctly rounded
  const double sc[8] = {-0x1.5555555555555p-3, 0x1.1111111111111p-7, -0x1.a01a01a01a01ap-13,
                        0x1.71de3a556c734p-19, -0x1.ae64567f544e4p-26, 0x1.6124613a86d09p-33,
                        -0x1.ae7f3e733b81fp-41, 0x1.952c77030ad4ap-49};
  const double cc[9] = {-0x1.0000000000000p-1, 0x1.5555555555555p-5, -0x1.6c16c16c16c17p-10,
                        0x1.a01a01a01a01ap-16, -0x1.27e4fb7789f5cp-22, 0x1.1eed8eff8d898p-29,
                        -0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-45, -0x1.6827863b97d97p-53};
  double p = sc[7];
#pragma unroll
  for (int i = 6; i >= 0; --i) p = __dadd_rn(__dmul_rn(p, s2), sc[i]);
  const double sin_t = __dadd_rn(t, __dmul_rn(__dmul_rn(t, s2), p));
  double q = cc[8];
#pragma unroll
  for (int i = 7; i >= 0; --i) q = __dadd_rn(__dmul_rn(q, s2), cc[i]);
  const double cos_t = __dadd_rn(1.0, __dmul_rn(s2, q));
  const bool swap = (k == 1) || (k == 2) || (k == 5) || (k == 6);
  const double ca = swap ? sin_t : cos_t;
  const double sa = swap ? cos_t : sin_t;
  *cs = (k >= 2 && k <= 5) ? -ca : ca;
  *sn = (k >= 4) ? -sa : sa;
}

// The four normals of Philox block `block` of (seed, problem, mode, stream).
__device__ __forceinline__ void gaussian4(uint64_t seed, uint64_t problem, uint64_t mode,
                                          uint64_t stream, uint64_t block, double z[4]) {
  uint64_t c[4] = {block, mode, problem, stream};
  philox4x64_10(c, seed, 0ull);
#pragma unroll
  for (int pair = 0; pair < 2; ++pair) {
    const double u1 = uniform_open01(c[2 * pair]);
    const double u2 = uniform_open01(c[2 * pair + 1]);
    const double r = __dsqrt_rn(__dmul_rn(-2.0, ln_open01(u1)));
    double cs, sn;
    sincos_2pi(u2, &cs, &sn);
    z[2 * pair] = __dmul_rn(r, cs);
    z[2 * pair + 1] = __dmul_rn(r, sn);
  }
}

// ---- float32 variant -------------------------------------------------------------------

__device__ __forceinline__ float uniform_open01_f32(uint64_t w) {
  return __fmul_rn(__fadd_rn(static_cast<float>(static_cast<uint32_t>(w >> 41)), 0.5f), 0x1p-23f);
}

// ln u, u in [2^-24, 1): reduction as in ln_open01, atanh series with 1/(2k+1), k = 1..5;
// e lies in [-23, 0], so e * ln2_hi (16 significant bits) is exact.
__device__ __forceinline__ float ln_open01_f32(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = static_cast<int>((bits >> 23) & 0xffu) - 126;
  float m = __uint_as_float((bits & 0x007fffffu) | 0x3f000000u);
  if (m < 0x1.6a09e6p-1f) {
    m = __fmul_rn(m, 2.0f);
    e -= 1;
  }
  const float f = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float s = __fmul_rn(f, f);
  const float c[5] = {0x1.555556p-2f, 0x1.99999ap-3f, 0x1.24924ap-3f, 0x1.c71c72p-4f, 0x1.745d18p-4f};
  float q = c[4];
#pragma unroll
  for (int k = 3; k >= 0; --k) q = __fadd_rn(__fmul_rn(q, s), c[k]);
  const float two_f = __fmul_rn(f, 2.0f);
  const float ln_m = __fadd_rn(two_f, __fmul_rn(__fmul_rn(two_f, s), q));
  const float ef = static_cast<float>(e);
  return __fadd_rn(__fmul_rn(ef, 0x1.62e4p-1f), __fadd_rn(__fmul_rn(ef, 0x1.7f7d1cp-20f), ln_m));
}

// (cos 2 pi u, sin 2 pi u) in float32; octant reduction as in sincos_2pi, Taylor terms
// (-1)^k/(2k+1)!, k = 1..4 and (-1)^k/(2k)!, k = 1..5.
__device__ __forceinline__ void sincos_2pi_f32(float u, float* cs, float* sn) {
  const float x = __fmul_rn(u, 8.0f);
  const float kf = floorf(x);
  const float f = __fsub_rn(x, kf);
  const int k = static_cast<int>(kf);
  const float g = (k & 1) ? __fsub_rn(1.0f, f) : f;
  const float t = __fmul_rn(g, 0x1.921fb6p-1f);
  const float s2 = __fmul_rn(t, t);
  const float sc[4] = {-0x1.555556p-3f, 0x1.111112p-7f, -0x1.a01a02p-13f, 0x1.71de3ap-19f};
  const float cc[5] = {-0x1p-1f, 0x1.555556p-5f, -0x1.6c16c2p-10f, 0x1.a01a02p-16f, -0x1.27e4fcp-22f};
  float p = sc[3];
#pragma unroll
  for (int i = 2; i >= 0; --i) p = __fadd_rn(__fmul_rn(p, s2), sc[i]);
  const float sin_t = __fadd_rn(t, __fmul_rn(__fmul_rn(t, s2), p));
  float q = cc[4];
#pragma unroll
  for (int i = 3; i >= 0; --i) q = __fadd_rn(__fmul_rn(q, s2), cc[i]);
  const float cos_t = __fadd_rn(1.0f, __fmul_rn(s2, q));
  const bool swap = (k == 1) || (k == 2) || (k == 5) || (k == 6);
  const float ca = swap ? sin_t : cos_t;
  const float sa = swap ? cos_t : sin_t;
  *cs = (k >= 2 && k <= 5) ? -ca : ca;
  *sn = (k >= 4) ? -sa : sa;
}

// The four float32 normals of Philox block `block` (same words and lanes as gaussian4).
__device__ __forceinline__ void gaussian4_f32(uint64_t seed, uint64_t problem, uint64_t mode,
                                              uint64_t stream, uint64_t block, float z[4]) {
  uint64_t c[4] = {block, mode, problem, stream};
  philox4x64_10(c, seed, 0ull);
#pragma unroll
  for (int pair = 0; pair < 2; ++pair) {
    const float u1 = uniform_open01_f32(c[2 * pair]);
    const float u2 = uniform_open01_f32(c[2 * pair + 1]);
    const float r = __fsqrt_rn(__fmul_rn(-2.0f, ln_open01_f32(u1)));
    float cs, sn;
    sincos_2pi_f32(u2, &cs, &sn);
    z[2 * pair] = __fmul_rn(r, cs);
    z[2 * pair + 1] = __fmul_rn(r, sn);
  }
}

// float32 -> bfloat16 (RNE), returned as the bfloat16 bit pattern.
__device__ __forceinline__ uint16_t f32_to_bf16_bits(float x) {
  uint32_t b = __float_as_uint(x);
  b = (b + 0x7FFFu + ((b >> 16) & 1u)) >> 16;
  return static_cast<uint16_t>(b);
}

__device__ __forceinline__ double bf16_bits_to_double(uint16_t h) {
  return static_cast<double>(__uint_as_float(static_cast<uint32_t>(h) << 16));
}

}  // namespace rng
}  // namespace tks

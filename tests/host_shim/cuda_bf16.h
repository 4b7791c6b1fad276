// Host stand-in for the CUDA header that the device RNG and the bf16 helpers include, for their CPU
// tests: correctly rounded IEEE operations as plain host arithmetic (built with -ffp-contract=off so
// that no multiply and add fuse), and bfloat16 as its 16-bit pattern with round-to-nearest-even from
// float32 written from the format's definition.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#define __device__
#define __forceinline__ inline

static inline uint64_t __umul64hi(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
}
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }
static inline double __dsqrt_rn(double a) { return sqrt(a); }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fdiv_rn(float a, float b) { return a / b; }
static inline float __fsqrt_rn(float a) { return sqrtf(a); }
static inline long long __double_as_longlong(double x) {
  long long r;
  memcpy(&r, &x, sizeof r);
  return r;
}
static inline double __longlong_as_double(long long x) {
  double r;
  memcpy(&r, &x, sizeof r);
  return r;
}
static inline uint32_t __float_as_uint(float x) {
  uint32_t r;
  memcpy(&r, &x, sizeof r);
  return r;
}
static inline float __uint_as_float(uint32_t x) {
  float r;
  memcpy(&r, &x, sizeof r);
  return r;
}

static inline float __double2float_rn(double a) { return (float)a; }

typedef struct {
  uint16_t x;
} __nv_bfloat16;

// float32 -> bfloat16, round to nearest, ties to even on the 16 dropped bits; NaN stays a quiet NaN
static inline __nv_bfloat16 __float2bfloat16_rn(float f) {
  uint32_t b = __float_as_uint(f);
  __nv_bfloat16 r;
  if ((b & 0x7fffffffu) > 0x7f800000u) {
    r.x = (uint16_t)((b >> 16) | 0x40u);
    return r;
  }
  b = (b + 0x7fffu + ((b >> 16) & 1u)) >> 16;
  r.x = (uint16_t)b;
  return r;
}
static inline uint16_t __bfloat16_as_ushort(__nv_bfloat16 h) { return h.x; }
static inline __nv_bfloat16 __ushort_as_bfloat16(uint16_t x) {
  __nv_bfloat16 r;
  r.x = x;
  return r;
}
static inline float __bfloat162float(__nv_bfloat16 h) { return __uint_as_float((uint32_t)h.x << 16); }

// Host stand-in for the CUDA header the device RNG includes: the RNG uses none of its types, only
// correctly rounded IEEE operations, which a host build provides here as plain arithmetic (built
// with -ffp-contract=off so that no multiply and add fuse).
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

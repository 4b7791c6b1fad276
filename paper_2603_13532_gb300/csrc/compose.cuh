// Rounding an exact integer sum to float64 without float64 instructions (host and device code; the
// host build is what the CPU tests check against exact rational rounding).
#pragma once

#include <stdint.h>
#include <string.h>
#ifndef __CUDACC__
#include <math.h>
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace tks {

// The level sums combine into the integer N = hi 2^28 + lo (hi, lo in 64 bits, |N| < 2^127), and the
// result is N 2^scale rounded once to nearest-even.  GB300's float64 pipe issues about 1.6 lanes per
// clock per SM against 64 or more for the integer pipes, so the epilogues build the float64 from the
// integer bits (leading-zero count, a 53-bit window with round/sticky bits, the exponent field)
// instead of converting and scaling in float64; results outside the normal range (never met by the
// products here) take a float64 path.
__host__ __device__ __forceinline__ int oz_clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ double oz_compose(long long hi, long long lo, int scale) {
  // 128-bit two's complement (nh, nl) of hi 2^28 + lo
  const unsigned long long h0 = (unsigned long long)hi << 28;
  const unsigned long long nl = h0 + (unsigned long long)lo;
  long long nh = (hi >> 36) + (lo < 0 ? -1 : 0) + (nl < h0 ? 1 : 0);
  const bool neg = nh < 0;
  unsigned long long ml = nl, mh = (unsigned long long)nh;
  if (neg) {
    ml = ~nl + 1ull;
    mh = ~mh + (ml == 0ull ? 1ull : 0ull);
  }
  if ((mh | ml) == 0ull) return 0.0;
  const int bitlen = mh ? 128 - oz_clz64(mh) : 64 - oz_clz64(ml);
  unsigned long long mant;
  int e2 = bitlen - 53;                       // |N| ~ mant 2^e2 with mant in [2^52, 2^53)
  if (e2 <= 0) {
    mant = ml << (-e2);
  } else {
    bool half, sticky;
    if (e2 < 64) {
      mant = (ml >> e2) | (e2 ? (mh << (64 - e2)) : 0ull);
      half = (ml >> (e2 - 1)) & 1ull;
      sticky = e2 > 1 ? (ml & ((1ull << (e2 - 1)) - 1ull)) != 0ull : false;
    } else {
      const int t = e2 - 64;
      mant = mh >> t;
      half = t ? ((mh >> (t - 1)) & 1ull) : (ml >> 63);
      sticky = t ? ((mh & ((1ull << (t - 1)) - 1ull)) != 0ull || ml != 0ull) : (ml << 1) != 0ull;
    }
    if (half && (sticky || (mant & 1ull))) ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++e2;
    }
  }
  const int field = e2 + 52 + scale + 1023;
  if (field >= 1 && field <= 2046) {
    const unsigned long long bits = (neg ? (1ull << 63) : 0ull) | ((unsigned long long)field << 52) |
                                    (mant & 0xfffffffffffffull);
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double d;
    memcpy(&d, &bits, sizeof(d));
    return d;
#endif
  }
  const double m = neg ? -(double)mant : (double)mant;
  return scalbn(m, e2 + scale);
}

// The same rounding for |hi|, |lo| < 2^60 (the digit products' level sums), without 128-bit
// arithmetic or branches: N = s 2^28 + r with s = hi + floor(lo / 2^28) and 0 <= r < 2^28, its
// magnitude m_hi 2^28 + m_lo (m_lo < 2^28), shifted right by k = max(bitlen(m_hi) - 36, 0) bits
// into one 64-bit word (the k bits shifted out only feed the sticky bit), then rounded to 53 bits.
__host__ __device__ __forceinline__ double oz_compose_b(long long hi, long long lo, int scale) {
  constexpr unsigned long long kMask28 = (1ull << 28) - 1ull;
  const long long sv = hi + (lo >> 28);
  const unsigned long long r = (unsigned long long)lo & kMask28;
  const bool neg = sv < 0;
  const unsigned long long mh = neg ? ~(unsigned long long)sv + (r == 0ull ? 1ull : 0ull) : (unsigned long long)sv;
  const unsigned long long ml = neg ? (0ull - r) & kMask28 : r;
  const int lh = 64 - oz_clz64(mh);
  const int k = lh > 36 ? lh - 36 : 0;
  const unsigned long long w = (mh << (28 - k)) | (ml >> k);
  const bool lost = (ml & ((1ull << k) - 1ull)) != 0ull;
  if (w == 0ull) return 0.0;
  const int lz = oz_clz64(w);
  const unsigned long long top = w << lz;               // leading one at bit 63
  unsigned long long mant = top >> 11;
  const bool half = (top >> 10) & 1ull;
  const bool sticky = lost || (top & 0x3ffull) != 0ull;
  mant += (half && (sticky || (mant & 1ull))) ? 1ull : 0ull;
  const int e_lead = 63 - lz + k + scale;               // exponent of N's leading bit, scaled
  const int field = e_lead + 1023;
  if (field >= 1 && field <= 2045) {
    // mant in [2^52, 2^53]: the implicit bit carries into the exponent field, so a mantissa that
    // rounded up to 2^53 gives the next binade with a zero fraction
    const unsigned long long bits = (neg ? (1ull << 63) : 0ull) + ((unsigned long long)(field - 1) << 52) + mant;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double d;
    memcpy(&d, &bits, sizeof(d));
    return d;
#endif
  }
  const double m = neg ? -(double)mant : (double)mant;
  return scalbn(m, e_lead - 52);
}

}  // namespace tks

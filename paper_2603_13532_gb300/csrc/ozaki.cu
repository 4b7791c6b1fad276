// Float64-accurate mode products on the tcgen05 tensor cores (the ST-HOSVD truncation of TKS_MIXED):
//   Y[l + L (c + rmax r)] = sum_a X[l + L (a + K r)] P[a + K c]      (H x_n P_n^T, and Q_n P_n)
//
// GB300 runs float64 FMAs at about 1 TFLOP/s against about 1.9 PFLOP/s for bf16 on the tensor pipe,
// so the product is computed from exact integer pieces (the Ozaki scheme, Ozaki, Ogita, Oishi and
// Rump 2012): every row of X and of P^T is scaled by a power of two 2^e bounding its entries and cut
// into eight signed 7-bit digits, x = 2^e sum_{s=1..8} d_s 2^(-7 s) + O(2^(e - 56)).  A digit is an
// integer in [-127, 127], exact in bfloat16; a digit product is exact; a sum of K <= 96 of them is
// an integer below 2^21, and the pairs of one level s + t (at most 8 pairs) below 2^24, so each level
// accumulates exactly in a float32 TMEM accumulator.  The epilogue adds the levels 2..9 in 64-bit
// integers and converts once:  y = 2^(eX + eP) sum_lambda A_lambda 2^(-7 lambda).  Dropping the
// levels above 9 and the digits beyond the eighth leaves an error of a few units of 2^-56 times the
// row maxima, the size of a float64 dot product's own rounding bound (K eps max|x| max|p|).
//
// Slicing runs on the integer pipe: the exponent, the significand and a shift from the float64 bits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "tc.cuh"

namespace tks {

namespace {

constexpr int kOzRowsPerCta = 32;
constexpr int kOzSliceThreads = 256;
constexpr int kOzMaxK = TKS_MAX_BASIS;

// ----------------------------------------------------------------------------- slicing
__global__ void __launch_bounds__(kOzSliceThreads) oz_slice_kernel(const OzSliceJob* __restrict__ jobs, int njobs,
                                                                  Bases bases) {
  __shared__ double xs[kOzRowsPerCta][kOzMaxK + 1];
  __shared__ int64_t roff[kOzRowsPerCta];
  __shared__ int rexp[kOzRowsPerCta];
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const OzSliceJob& J = jobs[lo];
  const int K = J.K;
  const int64_t L = J.L;
  const int64_t q0 = (int64_t)(blockIdx.x - J.tile_begin) * kOzRowsPerCta;
  const int nq = (int)(J.rows - q0 < kOzRowsPerCta ? J.rows - q0 : kOzRowsPerCta);
  const double* src = at<double>(bases, J.src);
  if (threadIdx.x < kOzRowsPerCta) {
    const int64_t q = q0 + threadIdx.x, r = q / L, l = q - r * L;
    roff[threadIdx.x] = l + L * (int64_t)K * r;
  }
  __syncthreads();
  // stage the rows, coalesced along a when L = 1 (rows contiguous), along the fibre index otherwise
  for (int e = threadIdx.x; e < kOzRowsPerCta * K; e += kOzSliceThreads) {
    int q, a;
    if (L == 1) { q = e / K; a = e - q * K; }
    else { a = e / kOzRowsPerCta; q = e - a * kOzRowsPerCta; }
    xs[q][a] = q < nq ? src[roff[q] + L * a] : 0.0;
  }
  __syncthreads();
  // row exponent e: |x| < 2^e for every entry (from the largest biased exponent field); 0 for a zero row
  {
    const int q = threadIdx.x >> 3, t8 = threadIdx.x & 7;
    int emax = 0;
    for (int a = t8; a < K; a += 8) {
      const int E = (int)((__double_as_longlong(xs[q][a]) >> 52) & 0x7ff);
      emax = E > emax ? E : emax;
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      const int other = __shfl_xor_sync(0xffffffffu, emax, o, 8);
      emax = other > emax ? other : emax;
    }
    if (t8 == 0) {
      const int e = emax == 0 ? 0 : (emax < 1 ? 1 : emax) - 1022;
      rexp[q] = e;
      if (q < nq) at<int32_t>(bases, J.expo)[q0 + q] = e;
    }
  }
  __syncthreads();
  uint16_t* planes = at<uint16_t>(bases, J.planes);
  const int64_t pstride = J.rows_pad * (int64_t)J.ld;
  for (int e = threadIdx.x; e < kOzRowsPerCta * K; e += kOzSliceThreads) {
    const int q = e / K, a = e - q * K;
    if (q >= nq) continue;
    const unsigned long long u = (unsigned long long)__double_as_longlong(xs[q][a]);
    const int E = (int)((u >> 52) & 0x7ff);
    const unsigned long long S = (u & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
    // M = floor(|x| 2^(56 - e)) = S 2^(Eeff - 1019 - e) < 2^56
    const int sh = (E ? E : 1) - 1019 - rexp[q];
    unsigned long long M = 0;
    if (sh >= 0) M = S << sh;
    else if (sh > -64) M = S >> (-sh);
    const bool neg = (u >> 63) != 0;
    uint16_t* out = planes + (q0 + q) * (int64_t)J.ld + a;
#pragma unroll
    for (int s = 0; s < kOzSlices; ++s) {
      const int d = (int)((M >> (49 - 7 * s)) & 127ull);
      out[s * pstride] = __bfloat16_as_ushort(__float2bfloat16_rn((float)(neg ? -d : d)));
    }
  }
}

// Digits of one float64 value against a row exponent e (|x| < 2^e): M = floor(|x| 2^(56 - e)) < 2^56
// from the exponent and significand bits, digit s = bits [49 - 7 s, 55 - 7 s] of M, signed as x.
__device__ __forceinline__ unsigned long long oz_magnitude(double x, int e, bool& neg) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7ff);
  const unsigned long long S = (u & 0xfffffffffffffull) | (E ? (1ull << 52) : 0ull);
  const int sh = (E ? E : 1) - 1019 - e;
  neg = (u >> 63) != 0;
  if (sh >= 0) return S << sh;
  return sh > -64 ? S >> (-sh) : 0ull;
}

__device__ __forceinline__ uint16_t oz_digit(unsigned long long M, int s, bool neg) {
  const int d = (int)((M >> (49 - 7 * s)) & 127ull);
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)(neg ? -d : d)));
}

// Column slicing for the Gram matrices of shifted CholeskyQR3: one CTA per column a of X (P rows),
// the column's exponent by a block reduction, then its digits along the row of each plane.
constexpr int kOzColThreads = 256;

__global__ void __launch_bounds__(kOzColThreads) oz_colslice_kernel(const OzColSliceJob* __restrict__ jobs,
                                                                   int njobs, Bases bases) {
  __shared__ int wmax[kOzColThreads / 32];
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const OzColSliceJob& J = jobs[lo];
  const int a = blockIdx.x - J.tile_begin;
  const int64_t P = J.P, L = J.L;
  const double* src = at<double>(bases, J.src);
  // element i = l + L r of column a at l + L a + L b r
  auto elem = [&](int64_t i) {
    const int64_t r = L == 1 ? i : i / L, l = i - r * L;
    return src[l + L * (int64_t)a + L * (int64_t)J.b * r];
  };
  int emax = 0;
  for (int64_t i = threadIdx.x; i < P; i += kOzColThreads) {
    const int E = (int)((__double_as_longlong(elem(i)) >> 52) & 0x7ff);
    emax = E > emax ? E : emax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int other = __shfl_xor_sync(0xffffffffu, emax, o);
    emax = other > emax ? other : emax;
  }
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = emax;
  __syncthreads();
  emax = 0;
  for (int w = 0; w < kOzColThreads / 32; ++w) emax = wmax[w] > emax ? wmax[w] : emax;
  const int e = emax == 0 ? 0 : emax - 1022;
  if (threadIdx.x == 0) at<int32_t>(bases, J.expo)[a] = e;
  uint16_t* planes = at<uint16_t>(bases, J.planes);
  const int64_t pstride = 64 * J.ldP;
  uint16_t* row = planes + (int64_t)a * J.ldP;
  for (int64_t i = threadIdx.x; i < P; i += kOzColThreads) {
    bool neg;
    const unsigned long long M = oz_magnitude(elem(i), e, neg);
#pragma unroll
    for (int sl = 0; sl < kOzSlices; ++sl) row[sl * pstride + i] = oz_digit(M, sl, neg);
  }
}

// ----------------------------------------------------------------------------- digit products
// One 128 x 64 tile of Y per CTA.  Warp 0 (one thread) loads the eight digit planes of the tile's X
// rows and of its P columns with TMA (one k-block of 64 at a time; K <= 96 takes two); warp 1 owns
// the kOzLevels TMEM accumulators (64 columns each, the whole 512) and one thread issues the 36
// digit-pair products of every k-block, pair (s, t) into accumulator s + t; warps 2-5 read the
// accumulators (TMEM lane quadrant warp % 4), combine the levels in 64-bit integers and write Y.
// Every wait is bounded: on a timeout the kernel records TKS_ETIMEOUT, drains its own copies and
// products (bounded), frees TMEM and returns.
constexpr int kOzBM = 128, kOzBN = 64, kOzBK = 64;
constexpr int kOzATile = kOzBM * kOzBK * 2;     // 16 KB per plane
constexpr int kOzBTile = kOzBN * kOzBK * 2;     // 8 KB per plane
constexpr size_t kOzSmem = 1024 + (size_t)kOzSlices * (kOzATile + kOzBTile) + 64;

__global__ void __launch_bounds__(192, 1) oz_gemm_kernel(const OzGemmJob* __restrict__ jobs, int njobs,
                                                       const CUtensorMap* __restrict__ maps, Bases bases,
                                                       Status* status, long long kOzWait) {
  extern __shared__ uint8_t oz_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(oz_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* At = smem;
  uint8_t* Bt = smem + kOzSlices * kOzATile;
  uint64_t* full = reinterpret_cast<uint64_t*>(Bt + kOzSlices * kOzBTile);
  uint64_t* empty = full + 1;
  uint64_t* tmem_full = empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_full + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const OzGemmJob& J = jobs[lo];
  const int local = blockIdx.x - J.tile_begin;
  const int tn = local % J.tiles_n, tm = local / J.tiles_n;
  const int m0 = tm * kOzBM, n0 = tn * kOzBN;
  const int nk = (J.K + kOzBK - 1) / kOzBK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    tc::mbar_init(full, 1);
    tc::mbar_init(empty, 1);
    tc::mbar_init(tmem_full, 1);
    *err = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, kOzLevels * kOzBN);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < kOzSlices; ++s) {
        tc::prefetch_tmap(&maps[J.mapA[s]]);
        tc::prefetch_tmap(&maps[J.mapB[s]]);
      }
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        // the single stage is refilled once the previous k-block's products have completed
        if (*err || !tc::mbar_wait(empty, (kb & 1) ^ 1, kOzWait)) {
          *err = 1;
          break;
        }
        tc::mbar_expect_tx(full, (uint32_t)(kOzSlices * (kOzATile + kOzBTile)));
        for (int s = 0; s < kOzSlices; ++s) {
          tc::tma_load_2d(At + s * kOzATile, &maps[J.mapA[s]], full, kb * kOzBK, m0);
          tc::tma_load_2d(Bt + s * kOzBTile, &maps[J.mapB[s]], full, kb * kOzBK, n0);
        }
        issued = kb + 1;
      }
      // drain: the last copies issued have landed before the CTA tears down
      if (issued > 0 && !tc::mbar_wait(full, (issued - 1) & 1, kOzWait)) *err = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kOzBM, kOzBN);
      for (int kb = 0; kb < nk; ++kb) {
        if (*err || !tc::mbar_wait(full, kb & 1, kOzWait)) {
          *err = 1;
          break;
        }
        tc::fence_after_sync();
        // level acc = s + t collects the digit pairs (s, t); its first product starts it at zero
        for (int acc = 0; acc < kOzLevels; ++acc) {
          const uint32_t d = tmem + (uint32_t)(acc * kOzBN);
          for (int s = 0; s <= acc; ++s) {
            const int t = acc - s;
            const uint32_t a0 = tc::smem_u32(At + s * kOzATile);
            const uint32_t b0 = tc::smem_u32(Bt + t * kOzBTile);
#pragma unroll
            for (int k = 0; k < kOzBK / 16; ++k) {
              const uint32_t accumulate = (kb > 0 || s > 0 || k > 0) ? 1u : 0u;
              tc::mma_bf16(d, tc::sw128_kmajor_desc(a0 + 32 * k), tc::sw128_kmajor_desc(b0 + 32 * k), idesc,
                           accumulate);
            }
          }
        }
        tc::mma_commit(empty);
      }
      tc::mma_commit(tmem_full);
      if (!tc::mbar_wait(tmem_full, 0, kOzWait)) *err = 1;
    }
  } else {
    bool ok = tc::mbar_wait(tmem_full, 0, kOzWait);
    ok = __all_sync(0xffffffffu, ok) && !*err;
    tc::fence_after_sync();
    if (ok) {
      const int q = warp & 3;
      const int row = m0 + 32 * q + lane;
      const bool live = row < J.M;
      const int eA = live ? at<const int32_t>(bases, J.expA)[row] : 0;
      const int32_t* expB = at<const int32_t>(bases, J.expB);
      double* Y = at<double>(bases, J.Y);
      const int64_t r = live ? (int64_t)row / J.L : 0, l = (int64_t)row - r * J.L;
      double* y = Y + l + J.L * (int64_t)J.rmax * r;
      for (int c0 = 0; c0 < kOzBN; c0 += 8) {
        uint32_t v[kOzLevels][8];
#pragma unroll
        for (int acc = 0; acc < kOzLevels; ++acc)
          tc::tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kOzBN + c0), v[acc]);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int col = n0 + c0 + j;
          if (!live || col >= J.N) continue;
          // exact integers below 2^24: sum_acc A_acc 2^(21 - 7 acc) in two 64-bit halves
          long long hi64 = 0, lo64 = 0;
#pragma unroll
          for (int acc = 0; acc < 4; ++acc)
            hi64 = (hi64 << 7) + (long long)__float2int_rn(__uint_as_float(v[acc][j]));
#pragma unroll
          for (int acc = 4; acc < kOzLevels; ++acc)
            lo64 = (lo64 << 7) + (long long)__float2int_rn(__uint_as_float(v[acc][j]));
          // value = 2^-35 (hi + 2^-28 lo), times 2^(eA + eB)
          const double val = fma((double)lo64, 3.7252902984619140625e-09, (double)hi64);
          y[J.L * (int64_t)col] = scalbn(val, eA + expB[col] - 35);
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, kOzLevels * kOzBN);
  if (threadIdx.x == 0 && *err) atomicCAS(&status->code, 0, (int)TKS_ETIMEOUT);
}

// ----------------------------------------------------------------------------- Gram matrices
// G = X^T X (b x b, b <= 64) from the column digit planes, one CTA per job.  Warp 0 (one thread) loads
// one k-block (64 rows of X) of all eight planes per stage, two stages; warp 1 owns the kOzLevels TMEM
// accumulators and issues the 36 digit-pair products per k-block with A and B the same 64-column tiles
// (an M = 128 product also reads the 64 rows after a tile, whose results land in TMEM lanes 64..127
// and are ignored).  Every kOzGramGroup k-blocks the level sums, exact integers (8 pairs x 128 x
// 127^2 < 2^24), are drained by warps 4 and 5 (TMEM lanes 0..63), combined in 64-bit integers and
// added in float64 into a shared-memory accumulator; the scale 2^(e_i + e_j) is applied once at the
// end.  Waits are bounded as in the other tensor-core kernels.
constexpr int kOzGramGroup = 2;
constexpr int kOzPlaneTile = 64 * kOzBK * 2;                          // 8 KB: 64 columns x 64 k
constexpr int kOzStageBytes = (kOzSlices + 1) * kOzPlaneTile;         // + the 8 KB an M = 128 read passes
constexpr size_t kOzGramSmem = 1024 + 2 * (size_t)kOzStageBytes + 64 * 64 * 8 + 128;

__global__ void __launch_bounds__(192, 1) oz_gram_kernel(const OzGramJob* __restrict__ jobs,
                                                       const CUtensorMap* __restrict__ maps, Bases bases,
                                                       Status* status, long long wait_cycles) {
  extern __shared__ uint8_t og_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(og_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage[2] = {smem, smem + kOzStageBytes};
  double* acc64 = reinterpret_cast<double*>(smem + 2 * kOzStageBytes);   // [row][col], 64 x 64
  uint64_t* full = reinterpret_cast<uint64_t*>(acc64 + 64 * 64);
  uint64_t* empty = full + 2;
  uint64_t* tmem_full = empty + 2;
  uint64_t* tmem_empty = tmem_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_empty + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const OzGramJob& J = jobs[blockIdx.x];
  const int nk = (int)((J.P + kOzBK - 1) / kOzBK);
  const int ngroups = (nk + kOzGramGroup - 1) / kOzGramGroup;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int st = 0; st < 2; ++st) {
      tc::mbar_init(&full[st], 1);
      tc::mbar_init(&empty[st], 1);
    }
    tc::mbar_init(tmem_full, 1);
    tc::mbar_init(tmem_empty, 2);
    *err = 0;
    tc::fence_barrier_init();
  }
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) acc64[e] = 0.0;
  if (warp == 1) tc::tmem_alloc(tmem_slot, kOzLevels * kOzBN);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      for (int sl = 0; sl < kOzSlices; ++sl) tc::prefetch_tmap(&maps[J.map[sl]]);
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        const int st = kb & 1, round = kb >> 1;
        if (*err || !tc::mbar_wait(&empty[st], (round & 1) ^ 1, wait_cycles)) {
          *err = 1;
          break;
        }
        tc::mbar_expect_tx(&full[st], (uint32_t)(kOzSlices * kOzPlaneTile));
        for (int sl = 0; sl < kOzSlices; ++sl)
          tc::tma_load_2d(stage[st] + sl * kOzPlaneTile, &maps[J.map[sl]], &full[st], kb * kOzBK, 0);
        issued = kb + 1;
      }
      // drain: every copy issued has landed before the CTA tears down
      for (int kb = (issued > 2 ? issued - 2 : 0); kb < issued; ++kb)
        if (!tc::mbar_wait(&full[kb & 1], (kb >> 1) & 1, wait_cycles)) *err = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kOzBM, kOzBN);
      for (int kb = 0; kb < nk; ++kb) {
        const int st = kb & 1, round = kb >> 1;
        const int g = kb / kOzGramGroup;
        const bool first = kb % kOzGramGroup == 0;
        const bool last = kb % kOzGramGroup == kOzGramGroup - 1 || kb == nk - 1;
        // a group starts once the previous group's sums have been drained
        if (first && g > 0 && (*err || !tc::mbar_wait(tmem_empty, (g - 1) & 1, wait_cycles))) {
          *err = 1;
          break;
        }
        if (*err || !tc::mbar_wait(&full[st], round & 1, wait_cycles)) {
          *err = 1;
          break;
        }
        tc::fence_after_sync();
        for (int acc = 0; acc < kOzLevels; ++acc) {
          const uint32_t d = tmem + (uint32_t)(acc * kOzBN);
          for (int sa = 0; sa <= acc; ++sa) {
            const uint32_t a0 = tc::smem_u32(stage[st] + sa * kOzPlaneTile);
            const uint32_t b0 = tc::smem_u32(stage[st] + (acc - sa) * kOzPlaneTile);
#pragma unroll
            for (int k = 0; k < kOzBK / 16; ++k) {
              const uint32_t accumulate = (!first || sa > 0 || k > 0) ? 1u : 0u;
              tc::mma_bf16(d, tc::sw128_kmajor_desc(a0 + 32 * k), tc::sw128_kmajor_desc(b0 + 32 * k), idesc,
                           accumulate);
            }
          }
        }
        tc::mma_commit(&empty[st]);
        if (last) tc::mma_commit(tmem_full);
      }
      // the last group's products have completed before teardown
      if (!*err && !tc::mbar_wait(tmem_full, (ngroups - 1) & 1, wait_cycles)) *err = 1;
    }
  } else if ((warp & 3) < 2) {
    // warps 4 and 5: TMEM lanes 0..63 (the rows of G)
    const int q = warp & 3;
    const int row = 32 * q + lane;
    for (int g = 0; g < ngroups; ++g) {
      bool ok = tc::mbar_wait(tmem_full, g & 1, wait_cycles);
      ok = __all_sync(0xffffffffu, ok) && !*err;
      if (!ok) {
        if (lane == 0) *err = 1;
        break;
      }
      tc::fence_after_sync();
      for (int c0 = 0; c0 < kOzBN; c0 += 8) {
        uint32_t v[kOzLevels][8];
#pragma unroll
        for (int acc = 0; acc < kOzLevels; ++acc)
          tc::tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kOzBN + c0), v[acc]);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          long long hi64 = 0, lo64 = 0;
#pragma unroll
          for (int acc = 0; acc < 4; ++acc)
            hi64 = (hi64 << 7) + (long long)__float2int_rn(__uint_as_float(v[acc][j]));
#pragma unroll
          for (int acc = 4; acc < kOzLevels; ++acc)
            lo64 = (lo64 << 7) + (long long)__float2int_rn(__uint_as_float(v[acc][j]));
          acc64[row * 64 + c0 + j] += fma((double)lo64, 3.7252902984619140625e-09, (double)hi64);
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tmem_empty);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, kOzLevels * kOzBN);
  if (!*err) {
    // G[i + b j] = 2^(e_i + e_j - 35) acc[i][j]
    const int32_t* expo = at<const int32_t>(bases, J.expo);
    double* G = at<double>(bases, J.G);
    const int b = J.b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int i = e % b, j = e / b;
      G[e] = scalbn(acc64[i * 64 + j], expo[i] + expo[j] - 35);
    }
  } else if (threadIdx.x == 0) {
    atomicCAS(&status->code, 0, (int)TKS_ETIMEOUT);
  }
}

}  // namespace

int oz_slice_tiles(int64_t rows) { return (int)((rows + kOzRowsPerCta - 1) / kOzRowsPerCta); }

void launch_oz_slice(const OzSliceJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream) {
  oz_slice_kernel<<<total_tiles, kOzSliceThreads, 0, stream>>>(jobs, njobs, bases);
}

cudaError_t prepare_oz_gemm() {
  cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(oz_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzGramSmem);
}

void launch_oz_colslice(const OzColSliceJob* jobs, int njobs, int total_cols, const Bases& bases,
                        cudaStream_t stream) {
  oz_colslice_kernel<<<total_cols, kOzColThreads, 0, stream>>>(jobs, njobs, bases);
}

void launch_oz_gram(const OzGramJob* jobs, int njobs, const void* maps, const Bases& bases, Status* status,
                    long long wait_cycles, cudaStream_t stream) {
  oz_gram_kernel<<<njobs, 192, kOzGramSmem, stream>>>(jobs, static_cast<const CUtensorMap*>(maps), bases, status,
                                                      wait_cycles);
}

void launch_oz_gemm(const OzGemmJob* jobs, int njobs, int total_tiles, const void* maps, const Bases& bases,
                    Status* status, long long wait_cycles, cudaStream_t stream) {
  oz_gemm_kernel<<<total_tiles, 192, kOzSmem, stream>>>(jobs, njobs, static_cast<const CUtensorMap*>(maps), bases,
                                                         status, wait_cycles);
}

}  // namespace tks

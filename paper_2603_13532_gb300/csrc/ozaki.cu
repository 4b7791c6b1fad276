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

#include "compose.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace tks {

namespace {

constexpr int kOzRowsPerCta = 32;
constexpr int kOzSliceThreads = 256;
constexpr int kOzMaxK = TKS_MAX_BASIS;

// ----------------------------------------------------------------------------- slicing
// bfloat16 bits of a digit d in [0, 127] carrying the sign of x, by full-rate integer and float32
// operations (the int -> float -> bfloat16 conversions run at a quarter of that rate): 2^23 + d is
// exact in float32, subtracting 2^23 leaves d, and d's float32 bits end in sixteen zeros.  Zero is +0.
__device__ __forceinline__ uint16_t oz_bf16_digit(int d, bool neg) {
  const float f = __int_as_float(0x4B000000 | d) - 8388608.0f;
  return (uint16_t)((__float_as_uint(f) >> 16) | ((neg && d) ? 0x8000u : 0u));
}

__global__ void __launch_bounds__(kOzSliceThreads) oz_slice_kernel(const OzSliceJob* __restrict__ jobs, int njobs,
                                                                  Bases bases) {
  __shared__ double xs[kOzRowsPerCta][kOzMaxK + 1];
  __shared__ int64_t roff[kOzRowsPerCta];
  __shared__ int rexp[kOzRowsPerCta];
  __shared__ int kx[kOzMaxK];      // per-column exponent offsets: element (q, a) is sliced as x 2^kx[a]
  const int lo = tile_job(jobs, njobs, (int)blockIdx.x);
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
  for (int a = threadIdx.x; a < K; a += kOzSliceThreads)
    kx[a] = J.kexp.base != B_NONE ? at<const int32_t>(bases, J.kexp)[a] : 0;
  __syncthreads();
  // stage the rows, coalesced along a when L = 1 (rows contiguous), along the fibre index otherwise
  for (int e = threadIdx.x; e < kOzRowsPerCta * K; e += kOzSliceThreads) {
    int q, a;
    if (L == 1) { q = e / K; a = e - q * K; }
    else { a = e / kOzRowsPerCta; q = e - a * kOzRowsPerCta; }
    xs[q][a] = q < nq ? src[roff[q] + L * a] : 0.0;
  }
  __syncthreads();
  // row exponent e: |x 2^kx| < 2^e for every entry (from the largest biased exponent field plus the
  // offset); 0 for a row without a normal entry
  {
    constexpr int kNone = -(1 << 20);
    const int q = threadIdx.x >> 3, t8 = threadIdx.x & 7;
    int emax = kNone;
    for (int a = t8; a < K; a += 8) {
      const int E = (int)((__double_as_longlong(xs[q][a]) >> 52) & 0x7ff);
      if (E) emax = E + kx[a] > emax ? E + kx[a] : emax;
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      const int other = __shfl_xor_sync(0xffffffffu, emax, o, 8);
      emax = other > emax ? other : emax;
    }
    if (t8 == 0) {
      const int e = emax == kNone ? 0 : emax - 1022;
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
    // M = floor(|x| 2^(kx + 56 - e)) = S 2^(Eeff + kx - 1019 - e) < 2^56
    const int sh = (E ? E : 1) - 1019 - (rexp[q] - kx[a]);
    unsigned long long M = 0;
    if (sh >= 0) M = S << sh;
    else if (sh > -64) M = S >> (-sh);
    const bool neg = (u >> 63) != 0;
    uint16_t* out = planes + (q0 + q) * (int64_t)J.ld + a;
#pragma unroll
    for (int s = 0; s < kOzSlices; ++s) {
      const int d = (int)((M >> (49 - 7 * s)) & 127ull);
      out[s * pstride] = oz_bf16_digit(d, neg);
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
  return oz_bf16_digit(d, neg);
}

// X of one CholeskyQR pass in 64-row tiles (one CTA per tile).  The tile is staged in shared memory
// with coalesced reads: rows are contiguous runs of b when L = 1, and for L > 1 each column of the
// tile is a run along l (crossing an r boundary at most where l wraps).
constexpr int kOzXRows = 64;
constexpr int kOzXThreads = 256;
constexpr int kOzXMaxB = 64;           // CholeskyQR3 runs for b <= 64
constexpr int kOzXPitch = 66;          // doubles per staged row; the same bytes hold 4 digit planes later

__device__ __forceinline__ const OzXSliceJob& oz_xjob(const OzXSliceJob* __restrict__ jobs, int njobs) {
  const int lo = tile_job(jobs, njobs, (int)blockIdx.x);
  return jobs[lo];
}

__device__ __forceinline__ int oz_stage_xtile(const OzXSliceJob& J, const double* __restrict__ src, int64_t i0,
                                              double (*xs)[kOzXPitch], int64_t* roff) {
  const int b = J.b;
  const int nq = (int)(J.P - i0 < kOzXRows ? J.P - i0 : kOzXRows);
  if (J.L == 1) {
    // the tile is nq * b contiguous values; the row index from a float32 reciprocal, exact for
    // e < 4096 and b <= 64 (the product stays 2^-22 away from the next integer)
    const double* base = src + i0 * b;
    const float rb = 1.0f / (float)b;
    for (int e = threadIdx.x; e < nq * b; e += kOzXThreads) {
      const int q = (int)(((float)e + 0.5f) * rb);
      xs[q][e - q * b] = base[e];
    }
  } else {
    if (threadIdx.x < kOzXRows) {
      const int64_t i = i0 + threadIdx.x, r = i / J.L, l = i - r * J.L;
      roff[threadIdx.x] = l + J.L * (int64_t)b * r;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kOzXRows * b; e += kOzXThreads) {
      const int a = e / kOzXRows, q = e - a * kOzXRows;
      if (q < nq) xs[q][a] = src[roff[q] + J.L * a];
    }
  }
  return nq;
}

__global__ void __launch_bounds__(kOzXThreads) oz_xmax_kernel(const OzXSliceJob* __restrict__ jobs, int njobs,
                                                             Bases bases) {
  __shared__ __align__(16) double xs[kOzXRows][kOzXPitch];
  __shared__ int64_t roff[kOzXRows];
  __shared__ int red[kOzXThreads / 64][64];
  const OzXSliceJob& J = oz_xjob(jobs, njobs);
  const int tile = blockIdx.x - J.tile_begin;
  const int nq = oz_stage_xtile(J, at<const double>(bases, J.src), (int64_t)tile * kOzXRows, xs, roff);
  __syncthreads();
  const int a = threadIdx.x & 63, g = threadIdx.x >> 6;
  int emax = 0;
  if (a < J.b)
    for (int q = g; q < nq; q += kOzXThreads / 64) {
      const int E = (int)((__double_as_longlong(xs[q][a]) >> 52) & 0x7ff);
      emax = E > emax ? E : emax;
    }
  red[g][a] = emax;
  __syncthreads();
  if (threadIdx.x < J.b) {
    int m = red[0][threadIdx.x];
    for (int k = 1; k < kOzXThreads / 64; ++k) m = red[k][threadIdx.x] > m ? red[k][threadIdx.x] : m;
    at<int32_t>(bases, J.part)[(int64_t)tile * 64 + threadIdx.x] = m;
  }
}

__global__ void __launch_bounds__(kOzXThreads) oz_xdig_kernel(const OzXSliceJob* __restrict__ jobs, int njobs,
                                                             Bases bases) {
  __shared__ __align__(16) double xs[kOzXRows][kOzXPitch];
  __shared__ int64_t roff[kOzXRows];
  __shared__ int red[kOzXThreads / 64][64];
  __shared__ int es[64];
  const OzXSliceJob& J = oz_xjob(jobs, njobs);
  const int tile = blockIdx.x - J.tile_begin;
  const int b = J.b;
  const int64_t i0 = (int64_t)tile * kOzXRows;
  // e_a = (largest biased exponent field of column a) - 1022, so |X[i][a]| < 2^e_a (0 for a zero column)
  {
    const int a = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int32_t* part = at<const int32_t>(bases, J.part);
    int m = 0;
    if (a < b)
      for (int t = g; t < J.tiles; t += kOzXThreads / 64) {
        const int v = part[(int64_t)t * 64 + a];
        m = v > m ? v : m;
      }
    red[g][a] = m;
  }
  const int nq = oz_stage_xtile(J, at<const double>(bases, J.src), i0, xs, roff);
  __syncthreads();
  if (threadIdx.x < b) {
    int m = red[0][threadIdx.x];
    for (int k = 1; k < kOzXThreads / 64; ++k) m = red[k][threadIdx.x] > m ? red[k][threadIdx.x] : m;
    const int e = m == 0 ? 0 : m - 1022;
    es[threadIdx.x] = e;
    if (tile == 0) at<int32_t>(bases, J.expo)[threadIdx.x] = e;
  }
  __syncthreads();
  uint16_t* colP = at<uint16_t>(bases, J.colP);
  const int64_t cstride = 64 * J.ldP;
  // each element's magnitude once, in registers (M < 2^56, the sign in bit 63; 0 outside the tile):
  // thread t holds column a = t % 64 of the row pairs (2 j, 2 j + 1), j = t / 64 + 4 k
  constexpr int kPairs = kOzXRows / 2 * 64 / kOzXThreads;   // 8 row pairs per thread
  const int a = threadIdx.x & 63, j0 = threadIdx.x >> 6;
  unsigned long long mg[kPairs][2];
#pragma unroll
  for (int k = 0; k < kPairs; ++k) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = 2 * (j0 + 4 * k) + h;
      mg[k][h] = 0ull;
      if (q < nq && a < b) {
        bool neg;
        const unsigned long long M = oz_magnitude(xs[q][a], es[a], neg);
        mg[k][h] = M | (neg ? (1ull << 63) : 0ull);
      }
    }
  }
  __syncthreads();
  // the staged tile's bytes now hold four digit planes at a time, as 32-bit words of two rows:
  // dg[s][j][a] = (digit of row 2 j + 1) << 16 | digit of row 2 j, rows of kDPitch words (an odd
  // count: the column reads below fall on distinct banks); each digit is formed once and leaves in
  // 16-byte stores of 8 rows of one column
  constexpr int kDPitch = 65;
  constexpr int kDPlane = kOzXRows / 2 * kDPitch;
  uint32_t* dg = reinterpret_cast<uint32_t*>(&xs[0][0]);
  static_assert(4 * kDPlane * sizeof(uint32_t) <= sizeof(xs), "four digit planes must fit the staged tile");
#pragma unroll
  for (int half = 0; half < 2; ++half) {
#pragma unroll
    for (int k = 0; k < kPairs; ++k) {
      const int j = j0 + 4 * k;
      // digits 0-3 are bits 28..55 of M and digits 4-7 bits 0..27: one 32-bit word per half; a zero
      // digit of a negative value becomes -0, which adds nothing to an exact sum
      const unsigned long long v0 = mg[k][0], v1 = mg[k][1];
      const uint32_t w0 = half == 0 ? (uint32_t)(v0 >> 28) & 0x0fffffffu : (uint32_t)v0 & 0x0fffffffu;
      const uint32_t w1 = half == 0 ? (uint32_t)(v1 >> 28) & 0x0fffffffu : (uint32_t)v1 & 0x0fffffffu;
      const uint32_t sg = ((uint32_t)(v0 >> 63) << 15) | ((uint32_t)(v1 >> 63) << 31);
#pragma unroll
      for (int s4 = 0; s4 < 4; ++s4) {
        const uint32_t d0 = (w0 >> (21 - 7 * s4)) & 127u, d1 = (w1 >> (21 - 7 * s4)) & 127u;
        // bf16 of a digit: the upper half of the float32 (2^23 + d) - 2^23, exact
        const float f0 = __int_as_float(0x4B000000 | (int)d0) - 8388608.0f;
        const float f1 = __int_as_float(0x4B000000 | (int)d1) - 8388608.0f;
        dg[s4 * kDPlane + j * kDPitch + a] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632) | sg;
      }
    }
    __syncthreads();
    // column planes: (slice, column a, 8 rows) -> one 16-byte store of plane row a
    for (int it = threadIdx.x; it < 4 * 64 * 8; it += kOzXThreads) {
      const int s4 = it >> 9, ac = (it >> 3) & 63, c = it & 7;
      if (ac < b && 8 * c < nq) {
        const uint32_t* src = dg + s4 * kDPlane + 4 * c * kDPitch + ac;
        const uint4 w = make_uint4(src[0], src[kDPitch], src[2 * kDPitch], src[3 * kDPitch]);
        *reinterpret_cast<uint4*>(colP + (4 * half + s4) * cstride + (int64_t)ac * J.ldP + i0 + 8 * c) = w;
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- digit products
// Persistent: CTA c takes the contiguous tile range [c T / G, (c + 1) T / G) of the T tiles (G CTAs,
// at most one per SM), so consecutive tiles mostly belong to one job and share its P digits.  Warp 0
// (one thread) loads the eight digit planes of a tile's X rows (and of its P columns when they change)
// with TMA, one k-block of 64 at a time (K <= 96 takes two); warp 1 owns the kOzLevels TMEM
// accumulators (64 columns each, the whole 512) and one thread issues the 36 digit-pair products of
// every k-block, pair (s, t) into accumulator s + t; warps 2-17 read the accumulators (TMEM lane
// quadrant warp % 4, columns 16 (warp - 2) / 4 ...), combine the levels in integers and write Y.
// Four epilogue warps per quadrant keep the integer pipes busy while one warp waits on a TMEM load.
// The next tile's planes load while the epilogue of the last one runs.  Every wait is bounded: on a
// timeout the kernel records TKS_ETIMEOUT, drains its own copies and products (bounded), frees TMEM
// and returns.
constexpr int kOzBM = 128, kOzBN = 64, kOzBK = 64;
constexpr int kOzATile = kOzBM * kOzBK * 2;     // 16 KB per plane
constexpr int kOzBTile = kOzBN * kOzBK * 2;     // 8 KB per plane
constexpr int kOzGemmThreads = 576;             // TMA, MMA and 16 epilogue warps
constexpr int kOzEpiCols = 16;                  // columns per epilogue warp
constexpr int kOzStagePitch = 5;                // staged stores: 32 rows x 4 columns (+1) per warp
constexpr size_t kOzSmem = 1024 + (size_t)kOzSlices * (kOzATile + kOzBTile) + 64 +
                           16 * 32 * kOzStagePitch * sizeof(double);

__device__ __forceinline__ int oz_tile_job(const OzGemmJob* __restrict__ jobs, int njobs, int t) {
  const int lo = tile_job(jobs, njobs, t);
  return lo;
}

__global__ void __launch_bounds__(kOzGemmThreads, 1) oz_gemm_kernel(const OzGemmJob* __restrict__ jobs, int njobs,
                                                                  int total_tiles,
                                                                  const CUtensorMap* __restrict__ maps, Bases bases,
                                                                  Status* status, long long kOzWait) {
  extern __shared__ uint8_t oz_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(oz_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* At = smem;
  uint8_t* Bt = smem + kOzSlices * kOzATile;
  // full/empty[h]: A planes 4h .. 4h + 3 of a k-block (half 0 also carries P's planes when they
  // change), so that the next tile's first half loads while the products of the second half run
  uint64_t* full = reinterpret_cast<uint64_t*>(Bt + kOzSlices * kOzBTile);
  uint64_t* empty = full + 2;
  uint64_t* tmem_full = empty + 2;
  uint64_t* tmem_empty = tmem_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_empty + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* ostage = reinterpret_cast<double*>(smem + kOzSlices * (kOzATile + kOzBTile) + 64);   // 16 x 32 x 5
  const int t_begin = (int)(((long long)blockIdx.x * total_tiles) / gridDim.x);
  const int t_end = (int)(((long long)(blockIdx.x + 1) * total_tiles) / gridDim.x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int h = 0; h < 2; ++h) {
      tc::mbar_init(&full[h], 1);
      tc::mbar_init(&empty[h], 1);
    }
    tc::mbar_init(tmem_full, 1);
    tc::mbar_init(tmem_empty, (kOzGemmThreads - 64) / 32);
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
      int issued = 0;        // k-blocks whose two halves were both issued
      int issued_h[2] = {0, 0};
      long long bkey = -1;   // (job, tile column, k-block) whose P planes are in shared memory
      for (int t = t_begin; t < t_end && !*err; ++t) {
        const int ji = oz_tile_job(jobs, njobs, t);
        const OzGemmJob& J = jobs[ji];
        const int local = t - J.tile_begin;
        const int tn = local % J.tiles_n, tm = local / J.tiles_n;
        const int nk = (J.K + kOzBK - 1) / kOzBK;
        if (t == t_begin || local == 0)
          for (int s = 0; s < kOzSlices; ++s) {
            tc::prefetch_tmap(&maps[J.mapA[s]]);
            tc::prefetch_tmap(&maps[J.mapB[s]]);
          }
        for (int kb = 0; kb < nk && !*err; ++kb) {
          const long long key = ((long long)ji << 24) | ((long long)tn << 4) | kb;
          const bool loadB = key != bkey;
          bkey = key;
          for (int h = 0; h < 2; ++h) {
            // half h is refilled once the previous k-block's products that read it have completed;
            // new P planes also wait for the second half (both halves' products read P)
            bool ok = tc::mbar_wait(&empty[h], (issued & 1) ^ 1, kOzWait);
            if (ok && h == 0 && loadB) ok = tc::mbar_wait(&empty[1], (issued & 1) ^ 1, kOzWait);
            if (*err || !ok) {
              *err = 1;
              break;
            }
            const bool withB = h == 0 && loadB;
            tc::mbar_expect_tx(&full[h], (uint32_t)(kOzSlices / 2 * kOzATile + (withB ? kOzSlices * kOzBTile : 0)));
            for (int s = 4 * h; s < 4 * h + 4; ++s) {
              if (J.a_mn) {
                // column planes: two 64-row boxes (rows fastest) per plane, K = 64 digit columns each
                tc::tma_load_2d(At + s * kOzATile, &maps[J.mapA[s]], &full[h], tm * kOzBM, kb * kOzBK);
                tc::tma_load_2d(At + s * kOzATile + kOzATile / 2, &maps[J.mapA[s]], &full[h], tm * kOzBM + kOzBM / 2,
                                kb * kOzBK);
              } else {
                tc::tma_load_2d(At + s * kOzATile, &maps[J.mapA[s]], &full[h], kb * kOzBK, tm * kOzBM);
              }
            }
            if (withB)
              for (int s = 0; s < kOzSlices; ++s)
                tc::tma_load_2d(Bt + s * kOzBTile, &maps[J.mapB[s]], &full[0], kb * kOzBK, tn * kOzBN);
            ++issued_h[h];
          }
          if (!*err) ++issued;
        }
      }
      // drain: the last copies issued into each half have landed before the CTA tears down
      for (int h = 0; h < 2; ++h)
        if (issued_h[h] > 0 && !tc::mbar_wait(&full[h], (issued_h[h] - 1) & 1, kOzWait)) *err = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc_k = tc::idesc_bf16_f32(kOzBM, kOzBN);
      constexpr uint32_t idesc_mn = tc::idesc_bf16_f32_amn(kOzBM, kOzBN);
      int used = 0, tiles = 0;
      for (int t = t_begin; t < t_end && !*err; ++t) {
        const OzGemmJob& J = jobs[oz_tile_job(jobs, njobs, t)];
        const int nk = (J.K + kOzBK - 1) / kOzBK;
        // the accumulators are free once the epilogue has read the previous tile
        if (!tc::mbar_wait(tmem_empty, (tiles & 1) ^ 1, kOzWait)) {
          *err = 1;
          break;
        }
        tc::fence_after_sync();
        bool ok = true;
        for (int kb = 0; kb < nk && ok; ++kb) {
          // level acc = s + t collects the digit pairs (s, t); its first product starts it at zero.
          // Plane descriptors once per k-block.  A 16-deep k step advances the start address by 32
          // bytes in a K-major tile (address field + 2) and by two 8-row groups, 2048 bytes, in an
          // MN-major one (+ 128); an MN-major A tile is two 64-row boxes 8 KB apart (LBO), 8-row
          // groups 1024 bytes apart (SBO).
          const bool amn = J.a_mn != 0;
          const uint32_t idesc = amn ? idesc_mn : idesc_k;
          const uint64_t astep = amn ? 128u : 2u;
          uint64_t dA[kOzSlices], dB[kOzSlices];
#pragma unroll
          for (int p = 0; p < kOzSlices; ++p) {
            const uint32_t sa = tc::smem_u32(At + p * kOzATile);
            dA[p] = amn ? tc::sw128_mnmajor_desc(sa, kOzATile / 2, 1024) : tc::sw128_kmajor_desc(sa);
            dB[p] = tc::sw128_kmajor_desc(tc::smem_u32(Bt + p * kOzBTile));
          }
          // first half: the pairs with s <= 3 (they start every level); second half: s >= 4
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (*err || !tc::mbar_wait(&full[h], used & 1, kOzWait)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
#pragma unroll
            for (int acc = 0; acc < kOzLevels; ++acc) {
              const uint32_t d = tmem + (uint32_t)(acc * kOzBN);
#pragma unroll
              for (int s = 4 * h; s <= acc && s < 4 * h + 4; ++s) {
#pragma unroll
                for (int k = 0; k < kOzBK / 16; ++k) {
                  const uint32_t accumulate = (kb > 0 || s > 0 || k > 0) ? 1u : 0u;
                  tc::mma_bf16(d, dA[s] + astep * k, dB[acc - s] + 2 * k, idesc, accumulate);
                }
              }
            }
            tc::mma_commit(&empty[h]);
          }
          if (ok) ++used;
        }
        if (!ok) {
          *err = 1;
          break;
        }
        tc::mma_commit(tmem_full);
        ++tiles;
      }
      // the last products have completed before TMEM is freed
      if (tiles > 0 && !tc::mbar_wait(tmem_full, (tiles - 1) & 1, kOzWait)) *err = 1;
    }
  } else {
    const int q = warp & 3;
    const int cbase = kOzEpiCols * ((warp - 2) >> 2);
    int tiles = 0;
    for (int t = t_begin; t < t_end; ++t) {
      // this tile's row and column exponents are read while the products run
      const OzGemmJob& J = jobs[oz_tile_job(jobs, njobs, t)];
      const int local = t - J.tile_begin;
      const int tn = local % J.tiles_n, tm = local / J.tiles_n;
      const int row = tm * kOzBM + 32 * q + lane;
      const bool live = row < J.M;
      const int n0 = tn * kOzBN + cbase;
      const int eA = (live && J.expA.base != B_NONE) ? at<const int32_t>(bases, J.expA)[row] : 0;
      const int ecol = n0 + (lane & (kOzEpiCols - 1));
      const int eB = ecol < J.N ? at<const int32_t>(bases, J.expB)[ecol] : 0;   // lane c: column n0 + c
      double* Y = at<double>(bases, J.Y);
      bool ok = tc::mbar_wait(tmem_full, tiles & 1, kOzWait);
      ok = __all_sync(0xffffffffu, ok) && !*err;
      if (!ok) {
        if (lane == 0) *err = 1;
        break;
      }
      tc::fence_after_sync();
      // this thread's row, columns n0 .. n0 + 15, composed before TMEM is released
      double outv[kOzEpiCols];
#pragma unroll
      for (int c0 = 0; c0 < kOzEpiCols; c0 += 4) {
        if (n0 + c0 < J.N) {   // warp-uniform
          uint32_t v[kOzLevels][4];
#pragma unroll
          for (int acc = 0; acc < kOzLevels; ++acc)
            tc::tmem_ld4(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kOzBN + cbase + c0), v[acc]);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // level sums are exact integers below 2^24, so adjacent levels pair exactly in 32 bits
            // (A_2i 2^7 + A_2i+1), and sum_acc A_acc 2^(49 - 7 acc) = hi 2^28 + lo with
            // hi = p0 2^14 + p1, lo = p2 2^14 + p3
            int p[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              p[i] = __float2int_rn(__uint_as_float(v[2 * i][j])) * 128 + __float2int_rn(__uint_as_float(v[2 * i + 1][j]));
            const long long hi64 = (long long)p[0] * 16384 + p[1];
            const long long lo64 = (long long)p[2] * 16384 + p[3];
            const int scale = eA + __shfl_sync(0xffffffffu, eB, c0 + j) - 63;
            // value = 2^-35 (hi + 2^-28 lo) 2^(eA + eB) = (hi 2^28 + lo) 2^(eA + eB - 63)
            outv[c0 + j] = (live && n0 + c0 + j < J.N) ? oz_compose_b(hi64, lo64, scale) : 0.0;
          }
        }
      }
      // every TMEM read of this tile has completed: the next tile's products may start
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tmem_empty);
      if (J.L == 1) {
        // rows are contiguous runs of rmax: transpose 32 rows x 4 columns through shared memory so
        // that each store covers eight rows' 32-byte segments instead of 32 scattered words
        double* st = ostage + (warp - 2) * (32 * kOzStagePitch);
        const int row0 = tm * kOzBM + 32 * q;
#pragma unroll
        for (int c0 = 0; c0 < kOzEpiCols; c0 += 4) {
          if (n0 + c0 < J.N) {
#pragma unroll
            for (int j = 0; j < 4; ++j) st[lane * kOzStagePitch + j] = outv[c0 + j];
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int r = 8 * i + (lane >> 2), c = lane & 3;
              const int rw = row0 + r, col = n0 + c0 + c;
              if (rw < J.M && col < J.N) Y[(int64_t)J.rmax * rw + col] = st[r * kOzStagePitch + c];
            }
            __syncwarp();
          }
        }
      } else if (live) {
        const int64_t r = (int64_t)row / J.L, l = (int64_t)row - r * J.L;
        double* y = Y + l + J.L * (int64_t)J.rmax * r;
#pragma unroll
        for (int c = 0; c < kOzEpiCols; ++c)
          if (n0 + c < J.N) y[J.L * (int64_t)(n0 + c)] = outv[c];
      }
      ++tiles;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, kOzLevels * kOzBN);
  if (threadIdx.x == 0 && *err) atomicCAS(&status->code, 0, (int)TKS_ETIMEOUT);
}

// ----------------------------------------------------------------------------- Gram matrices
// G = X^T X (b x b, b <= 64) from the column digit planes, one CTA per job.  Warp 0 (one thread) loads
// one k-block (64 rows of X) of all eight planes per stage, two stages, each plane a 64-column tile,
// stored in the order 0, 4, 1, 5, 2, 6, 3, 7 so that planes s and s + 4 form one 128-row operand.
// Warp 1 issues, per k-block, the 26 products [X_s; X_(s+4)]^T X_t (s <= 3, s + t <= 7) into TMEM
// block s + t: lanes 0..63 collect the digit pair (s, t) at level s + t, lanes 64..127 the pair
// (s + 4, t) at level s + t + 4 (used for blocks 0..3, where s + t + 4 <= 7; the rest is ignored), so
// the 36 pairs of levels 0..7 take 26 M = 128 products.  A level sum holds at most 4 pairs per block,
// so kOzGramGroup = 4 k-blocks stay exact integers in float32 (4 pairs x 256 x 127^2 < 2^24); after
// each group warps 4, 5, 8, 9 (TMEM lanes 0..63: levels 0..7 of the pairs s <= 3) and warps 2, 3, 6, 7
// (lanes 64..127: levels 4..7 of the pairs s >= 4) combine the levels in integers and add them into
// 64-bit integer accumulators in shared memory (hi, lo and the upper lanes' lo), so G is the exact
// sum rounded once at the end, with the scale 2^(e_i + e_j).  Waits are bounded as in the other
// tensor-core kernels.
constexpr int kOzGramGroup = 4;
constexpr int kOzGramThreads = 320;   // TMA, MMA, and drain warps 2..9 (two per TMEM lane quadrant)
constexpr int kOzPlaneTile = 64 * kOzBK * 2;                          // 8 KB: 64 columns x 64 k
constexpr int kOzStageBytes = kOzSlices * kOzPlaneTile;
constexpr size_t kOzGramSmem = 1024 + 2 * (size_t)kOzStageBytes + 3 * 64 * 64 * 8 + 128;

__device__ __forceinline__ int oz_gram_pos(int plane) { return plane < 4 ? 2 * plane : 2 * (plane - 4) + 1; }

__global__ void __launch_bounds__(kOzGramThreads, 1) oz_gram_kernel(const OzGramJob* __restrict__ jobs,
                                                       const CUtensorMap* __restrict__ maps, Bases bases,
                                                       Status* status, long long wait_cycles) {
  extern __shared__ uint8_t og_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(og_smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage[2] = {smem, smem + kOzStageBytes};
  // the level sums of every drain, combined exactly in 64-bit integers per entry, [col][row]:
  // hi (levels 0..3) and lo (levels 4..7) of the pairs s <= 3, lo2 (levels 4..7) of the pairs s >= 4
  long long* acc_hi = reinterpret_cast<long long*>(smem + 2 * kOzStageBytes);
  long long* acc_lo = acc_hi + 64 * 64;
  long long* acc_lo2 = acc_lo + 64 * 64;
  uint64_t* full = reinterpret_cast<uint64_t*>(acc_lo2 + 64 * 64);
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
    tc::mbar_init(tmem_empty, 8);
    *err = 0;
    tc::fence_barrier_init();
  }
  for (int e = threadIdx.x; e < 3 * 64 * 64; e += blockDim.x) acc_hi[e] = 0;
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
          tc::tma_load_2d(stage[st] + oz_gram_pos(sl) * kOzPlaneTile, &maps[J.map[sl]], &full[st], kb * kOzBK, 0);
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
        // plane descriptors once per k-block (a 16-deep k step adds 2 to the address field); the
        // 128-row operand of plane s <= 3 starts at its tile and runs on into plane s + 4's
        uint64_t dP[kOzSlices];
#pragma unroll
        for (int p = 0; p < kOzSlices; ++p)
          dP[p] = tc::sw128_kmajor_desc(tc::smem_u32(stage[st] + oz_gram_pos(p) * kOzPlaneTile));
#pragma unroll
        for (int blk = 0; blk < kOzLevels; ++blk) {
          const uint32_t d = tmem + (uint32_t)(blk * kOzBN);
#pragma unroll
          for (int sa = 0; sa <= blk && sa < 4; ++sa) {
#pragma unroll
            for (int k = 0; k < kOzBK / 16; ++k) {
              const uint32_t accumulate = (!first || sa > 0 || k > 0) ? 1u : 0u;
              tc::mma_bf16(d, dP[sa] + 2 * k, dP[blk - sa] + 2 * k, idesc, accumulate);
            }
          }
        }
        tc::mma_commit(&empty[st]);
        if (last) tc::mma_commit(tmem_full);
      }
      // the last group's products have completed before teardown
      if (!*err && !tc::mbar_wait(tmem_full, (ngroups - 1) & 1, wait_cycles)) *err = 1;
    }
  } else {
    // warps 4, 5, 8, 9: TMEM lanes 0..63, blocks 0..7; warps 2, 3, 6, 7: lanes 64..127, blocks 0..3.
    // Warps 2..5 take columns 0..31, warps 6..9 columns 32..63.
    const int q = warp & 3;
    const bool upper = q >= 2;
    const int row = 32 * (q & 1) + lane;   // the row of G (column of X) this lane holds
    const int cb = warp >= 6 ? 32 : 0;
    for (int g = 0; g < ngroups; ++g) {
      bool ok = tc::mbar_wait(tmem_full, g & 1, wait_cycles);
      ok = __all_sync(0xffffffffu, ok) && !*err;
      if (!ok) {
        if (lane == 0) *err = 1;
        break;
      }
      tc::fence_after_sync();
      const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
      for (int c0 = cb; c0 < cb + 32 && c0 < J.b; c0 += 8) {
        if (!upper) {
          uint32_t v[kOzLevels][8];
#pragma unroll
          for (int blk = 0; blk < kOzLevels; ++blk) tc::tmem_ld8(tl + (uint32_t)(blk * kOzBN + c0), v[blk]);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // exact integers below 2^24: adjacent levels pair in 32 bits, then hi = p0 2^14 + p1,
            // lo = p2 2^14 + p3 (sum_L A_L 2^(49 - 7 L) = hi 2^28 + lo)
            int p[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              p[i] = __float2int_rn(__uint_as_float(v[2 * i][j])) * 128 + __float2int_rn(__uint_as_float(v[2 * i + 1][j]));
            acc_hi[(c0 + j) * 64 + row] += (long long)p[0] * 16384 + p[1];
            acc_lo[(c0 + j) * 64 + row] += (long long)p[2] * 16384 + p[3];
          }
        } else {
          // block L - 4 of these lanes holds level L = 4..7 of the pairs s >= 4
          uint32_t v[4][8];
#pragma unroll
          for (int blk = 0; blk < 4; ++blk) tc::tmem_ld8(tl + (uint32_t)(blk * kOzBN + c0), v[blk]);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int p2 = __float2int_rn(__uint_as_float(v[0][j])) * 128 + __float2int_rn(__uint_as_float(v[1][j]));
            const int p3 = __float2int_rn(__uint_as_float(v[2][j])) * 128 + __float2int_rn(__uint_as_float(v[3][j]));
            acc_lo2[(c0 + j) * 64 + row] += (long long)p2 * 16384 + p3;
          }
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
    // G[i + b j] = (hi 2^28 + lo + lo2) 2^(e_i + e_j - 63), rounded once
    const int32_t* expo = at<const int32_t>(bases, J.expo);
    double* G = at<double>(bases, J.G);
    const int b = J.b;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int i = e % b, j = e / b;
      G[e] = oz_compose(acc_hi[j * 64 + i], acc_lo[j * 64 + i] + acc_lo2[j * 64 + i], expo[i] + expo[j] - 63);
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

int oz_xslice_tiles(int64_t rows) { return (int)((rows + kOzXRows - 1) / kOzXRows); }

void launch_oz_xmax(const OzXSliceJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream) {
  oz_xmax_kernel<<<total_tiles, kOzXThreads, 0, stream>>>(jobs, njobs, bases);
}

void launch_oz_xdig(const OzXSliceJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream) {
  oz_xdig_kernel<<<total_tiles, kOzXThreads, 0, stream>>>(jobs, njobs, bases);
}

void launch_oz_gram(const OzGramJob* jobs, int njobs, const void* maps, const Bases& bases, Status* status,
                    long long wait_cycles, cudaStream_t stream) {
  oz_gram_kernel<<<njobs, kOzGramThreads, kOzGramSmem, stream>>>(jobs, static_cast<const CUtensorMap*>(maps), bases, status,
                                                      wait_cycles);
}

void launch_oz_gemm(const OzGemmJob* jobs, int njobs, int total_tiles, const void* maps, const Bases& bases,
                    Status* status, long long wait_cycles, cudaStream_t stream) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms <= 0)
      sms = 148;
  }
  const int grid = total_tiles < sms ? total_tiles : sms;
  if (grid <= 0) return;
  oz_gemm_kernel<<<grid, kOzGemmThreads, kOzSmem, stream>>>(jobs, njobs, total_tiles,
                                                             static_cast<const CUtensorMap*>(maps), bases, status,
                                                             wait_cycles);
}

}  // namespace tks

// Khatri-Rao core sketches of an order-3 term with the tcgen05 tensor cores (mixed-precision path).
//
// Alg. 4 (KRPSum-Tucker), Sec. 3.1.1: with M_m = U_k^(m)T Omega_m (r_m x s) the sketch of mode n is
// V_kn = G_k,(n) (M_l (.) M_j) (r_n x s), {j, l} the other two modes: column c of V_kn is the core
// contracted with column c of M_j and of M_l.  One CTA per term computes it in two stages per mode:
//   Z[(i_n, i_j), c] = sum_{i_l} G[i_n, i_j, i_l] M_l[i_l, c]        (tensor cores)
//   V_kn[i_n, c]     = sum_{i_j} Z[(i_n, i_j), c] M_j[i_j, c]         (CUDA cores, per column c)
// with (j, l) = (1, 2), (0, 2), (0, 1) for n = 0, 1, 2.  The first stage is a product with M = 128
// rows (i_n, i_j) per tile (i_n padded to a power of two P, row = i_n + P (i_j - i_j0)), N = 64
// columns c and K = r_l (padded to 16 or 32): A is the core, exact in bfloat16, gathered from a copy
// of the core in shared memory ordered (i_n, i_j, i_l) (the stored order for n = 0; for n = 1, 2 a
// transposed copy with an odd row stride, made from the stored one); B is M_l^T split exactly into three bf16
// planes (hi + mid + lo = the float32 value), so the three plane products reproduce the float32
// contraction to float32 rounding.  One elected thread issues them into one of two TMEM
// accumulators of 64 columns; while the next tile's A is gathered, all eight warps read the last
// accumulator back (warp w: TMEM lanes 32 (w % 4) .., columns 32 (w / 4) ..) and add Z M_j into
// per-thread sums for their row's i_n, which are reduced across rows through shared memory at the
// end of the mode and written, scaled by alpha_k, as the three bf16 planes of V_kn.  Every wait is
// bounded: on a timeout the kernel records TKS_ETIMEOUT, waits (bounded) for its products in flight,
// frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fastdiv.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace tks {

namespace {

constexpr int kThreads = 256;
constexpr int kCols = 64;                   // sketch columns (s <= 64): N of the products
constexpr int kMaxR = kSketch3MaxRank;      // 32
constexpr int kRows = 128;                  // M of the products
// K-major operand tiles without swizzle: 8-row x 16-byte core matrices; the k blocks of a row group
// kLbo bytes apart, row groups kp / 8 * kLbo bytes apart (kp = 16 or 32).
constexpr int kLbo = 128;
constexpr int kATile = kRows * kMaxR * 2;   // 8 KB: 128 rows x 32 k
constexpr int kBPlane = kCols * kMaxR * 2;  // 4 KB: 64 rows x 32 k
constexpr int kRedLd = kCols + 1;           // row stride (floats) of the reduction buffer
// Layout: M_0..M_2 ([m][i][c] float32, zero outside i < r_m, c < s), two A stages, three B planes,
// the core as stored, then the transposed copy of the current mode, which the end-of-mode reduction
// ([row][c]) overwrites.
constexpr int kMOff = 0;
constexpr int kAOff = kMOff + 3 * kMaxR * kCols * (int)sizeof(float);
constexpr int kBOff = kAOff + 2 * kATile;
constexpr int kGOff = kBOff + 3 * kBPlane;
constexpr int kRedBytes = kRows * kRedLd * (int)sizeof(float);
constexpr int kTmemCols = 128;
constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

__device__ __forceinline__ int tile_offset(int row, int k, int kp) {
  return (row >> 3) * (kp / 8) * kLbo + (k >> 3) * kLbo + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// v = hi + mid + lo exactly, each part a bfloat16 (returned in the upper 16 bits): hi is v truncated
// to its leading 8 significant bits, mid the same of the remainder, lo the rest (at most 8
// significant bits).  Masks and exact float32 subtractions: no conversion instructions.
__device__ __forceinline__ void split3_exact(float v, uint32_t& u0, uint32_t& u1, uint32_t& u2) {
  u0 = __float_as_uint(v) & 0xffff0000u;
  const float r1 = v - __uint_as_float(u0);
  u1 = __float_as_uint(r1) & 0xffff0000u;
  u2 = __float_as_uint(r1 - __uint_as_float(u1));
}

__global__ void __launch_bounds__(kThreads) sketch3_tc_kernel(const Sketch3Job* __restrict__ jobs, Bases bases,
                                                              Status* status) {
  extern __shared__ __align__(16) unsigned char sk_smem[];
  __shared__ uint64_t full[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int err;
  const Sketch3Job& J = jobs[blockIdx.x];
  const int r0 = J.r[0], r1 = J.r[1], r2 = J.r[2];
  const int s = J.s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float* Ms = reinterpret_cast<float*>(sk_smem + kMOff);
  unsigned char* Ast = sk_smem + kAOff;
  unsigned char* Bp = sk_smem + kBOff;
  const int tot = r0 * r1 * r2;
  const int tpad = (2 * tot + 15) & ~15;
  uint16_t* Gs = reinterpret_cast<uint16_t*>(sk_smem + kGOff);
  uint16_t* Gx = reinterpret_cast<uint16_t*>(sk_smem + kGOff + tpad);
  float* red = reinterpret_cast<float*>(sk_smem + kGOff + tpad);
  const uint16_t* G = at<uint16_t>(bases, J.core);

  if (tid == 0) {
    tc::mbar_init(&full[0], 1);
    tc::mbar_init(&full[1], 1);
    err = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc(&tmem_slot, kTmemCols);
  for (int m = 0; m < 3; ++m) {
    const float* Mg = at<float>(bases, J.M[m]) + J.roff[m];
    const int rm = m == 0 ? r0 : (m == 1 ? r1 : r2);
    for (int e = tid; e < kMaxR * kCols; e += kThreads) {
      const int i = e >> 6, c = e & (kCols - 1);
      Ms[m * kMaxR * kCols + e] = (i < rm && c < s) ? Mg[i + (int64_t)J.R[m] * c] : 0.f;
    }
  }
  for (int e0 = 0; e0 < tot; e0 += 8 * kThreads) {
    uint16_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kThreads + tid;
      v[u] = e < tot ? G[e] : (uint16_t)0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kThreads + tid;
      if (e < tot) Gs[e] = v[u];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  int g = 0;   // products issued so far (tiles over all modes): buffer g & 1, phase (g >> 1) & 1
  for (int n = 0; n < 3 && !err; ++n) {
    const int j = n == 0 ? 1 : 0, l = n == 2 ? 1 : 2;
    const int rn = n == 0 ? r0 : (n == 1 ? r1 : r2);
    const int rj = j == 0 ? r0 : r1;
    const int rl = l == 1 ? r1 : r2;
    int pb = 0;
    while ((1 << pb) < rn) ++pb;                 // P = 2^pb >= r_n
    const int per = kRows >> pb;                 // i_j per tile
    const int tiles = (rj + per - 1) / per;
    const int kp = rl <= 16 ? 16 : 32;
    const float* Mj = Ms + j * kMaxR * kCols;
    const float* Ml = Ms + l * kMaxR * kCols;
    const SmallDiv drn(rn);
    // the core ordered (i_n, i_j, i_l), i_n fastest: Gt[i_n + ld (i_j + r_j i_l)] -- the stored core
    // for n = 0 (ld = r_0); for n = 1, 2 a copy with ld = r_n | 1 (odd: the copy's strided stores fall
    // on distinct banks), made with one thread per (i_j, i_l), whose reads of the stored core
    // (i_j = i_0 fastest) are consecutive across a warp
    const uint16_t* Gt = Gs;
    int ld = r0;
    if (n > 0) {
      ld = rn | 1;
      const int outer = rj * rl;           // o = i_0 + r_0 i_l
      const int step = n == 1 ? r0 : r0 * r1;   // stored-core stride of i_n
      for (int o = tid; o < outer; o += kThreads) {
        const int il = o / r0, i0 = o - il * r0;
        const uint16_t* src = Gs + i0 + (n == 1 ? r0 * r1 * il : r0 * il);
        uint16_t* dst = Gx + ld * o;
        for (int in = 0; in < rn; ++in) dst[in] = src[step * in];
      }
      Gt = Gx;
    }
    // B: planes of M_l^T (rows c, k = i_l < kp; zero for k >= r_l), one 8-k block per thread
    for (int item = tid; item < kCols * (kp / 8); item += kThreads) {
      const int c = item & (kCols - 1), kb = item >> 6;
      uint32_t p0[4], p1[4], p2[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        uint32_t a0, a1, a2, b0, b1, b2;
        split3_exact(Ml[(8 * kb + 2 * e) * kCols + c], a0, a1, a2);
        split3_exact(Ml[(8 * kb + 2 * e + 1) * kCols + c], b0, b1, b2);
        p0[e] = __byte_perm(a0, b0, 0x7632);
        p1[e] = __byte_perm(a1, b1, 0x7632);
        p2[e] = __byte_perm(a2, b2, 0x7632);
      }
      const int off = tile_offset(c, 8 * kb, kp);
      *reinterpret_cast<uint4*>(Bp + off) = make_uint4(p0[0], p0[1], p0[2], p0[3]);
      *reinterpret_cast<uint4*>(Bp + kBPlane + off) = make_uint4(p1[0], p1[1], p1[2], p1[3]);
      *reinterpret_cast<uint4*>(Bp + 2 * kBPlane + off) = make_uint4(p2[0], p2[1], p2[2], p2[3]);
    }
    __syncthreads();   // the transposed copy is complete before any thread gathers from it
    // this thread's row of every tile and its 32 columns of the read-back
    const int q = warp & 3, h = warp >> 2;
    const int rho = 32 * q + lane;
    const int jr = rho >> pb;
    float acc[32];
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) acc[cc] = 0.f;

    for (int t = 0; t <= tiles; ++t) {
      if (t < tiles) {
        // A(t): rows = i_n + P (i_j - per t), k = i_l; zero outside the core
        unsigned char* A = Ast + (g & 1) * kATile;
        for (int item = tid; item < kRows * (kp / 8); item += kThreads) {
          const int row = item & (kRows - 1), kb = item >> 7;
          const int in = row & ((1 << pb) - 1), ij = per * t + (row >> pb);
          const bool live = in < rn && ij < rj;
          const int base = in + ld * ij;
          uint16_t v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int il = 8 * kb + e;
            const bool ok = live && il < rl;
            const uint16_t gv = Gt[ok ? base + ld * rj * il : 0];
            v[e] = ok ? gv : (uint16_t)0;
          }
          *reinterpret_cast<uint4*>(A + tile_offset(row, 8 * kb, kp)) =
              make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
        }
        tc::fence_proxy_async_smem();
      }
      tc::fence_before_sync();
      __syncthreads();   // A(t) is complete; every read of the accumulator MMA(t) reuses has finished
      tc::fence_after_sync();
      if (err) break;
      if (t < tiles && tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(kRows, kCols);
        const uint32_t d = tmem + (uint32_t)(kCols * (g & 1));
        const uint32_t a0 = tc::smem_u32(Ast + (g & 1) * kATile), b0 = tc::smem_u32(Bp);
        const uint32_t sbo = (uint32_t)(kp / 8 * kLbo);
        for (int ks = 0; ks < kp / 16; ++ks) {
          const uint64_t da = tc::plain_kmajor_desc(a0 + 2 * kLbo * ks, kLbo, sbo);
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            const uint64_t db = tc::plain_kmajor_desc(b0 + p * kBPlane + 2 * kLbo * ks, kLbo, sbo);
            tc::mma_bf16(d, da, db, idesc, (ks > 0 || p > 0) ? 1u : 0u);
          }
        }
        tc::mma_commit(&full[g & 1]);
      }
      if (t >= 1) {
        // read back Z(t - 1) and add Z M_j into this row's sums
        const int gp = g - 1;
        const bool ok = tc::mbar_wait(&full[gp & 1], (gp >> 1) & 1, kWaitCycles);
        if (!__all_sync(0xffffffffu, ok)) {
          if (lane == 0) err = 1;
        } else {
          tc::fence_after_sync();
          uint32_t v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kCols * (gp & 1) + 32 * h), v);
          tc::tmem_ld_wait();
          const int ij = per * (t - 1) + jr;
          if (ij < rj) {
            const float4* mj = reinterpret_cast<const float4*>(Mj + ij * kCols + 32 * h);
#pragma unroll
            for (int c4 = 0; c4 < 8; ++c4) {
              const float4 w = mj[c4];
              acc[4 * c4] = fmaf(__uint_as_float(v[4 * c4]), w.x, acc[4 * c4]);
              acc[4 * c4 + 1] = fmaf(__uint_as_float(v[4 * c4 + 1]), w.y, acc[4 * c4 + 1]);
              acc[4 * c4 + 2] = fmaf(__uint_as_float(v[4 * c4 + 2]), w.z, acc[4 * c4 + 2]);
              acc[4 * c4 + 3] = fmaf(__uint_as_float(v[4 * c4 + 3]), w.w, acc[4 * c4 + 3]);
            }
          }
        }
      }
      if (t < tiles) ++g;
    }
    __syncthreads();   // a timeout recorded by the last read-back is seen by every thread
    if (err) break;
    // V_kn[i_n, c] = alpha sum over the rows i_n + P m of their sums (the transposed copy is no
    // longer read)
#pragma unroll
    for (int cc = 0; cc < 32; ++cc) red[rho * kRedLd + 32 * h + cc] = acc[cc];
    __syncthreads();
    {
      uint16_t* P0 = at<uint16_t>(bases, J.V[n][0]);
      uint16_t* P1 = at<uint16_t>(bases, J.V[n][1]);
      uint16_t* P2 = at<uint16_t>(bases, J.V[n][2]);
      const int groups = kRows >> pb;
      for (int e = tid; e < rn * kCols; e += kThreads) {
        const int c = drn.quo(e), in = e - c * rn;   // consecutive threads: consecutive i_n of a column
        if (c < s) {
          float sum = 0.f;
          for (int m = 0; m < groups; ++m) sum += red[(in + (m << pb)) * kRedLd + c];
          uint32_t u0, u1, u2;
          split3_exact(J.alpha * sum, u0, u1, u2);
          const int64_t o = J.roff[n] + in + (int64_t)J.ldv[n] * c;
          P0[o] = (uint16_t)(u0 >> 16);
          P1[o] = (uint16_t)(u1 >> 16);
          P2[o] = (uint16_t)(u2 >> 16);
        }
      }
    }
    __syncthreads();   // the reduction buffer is read before the next mode's transposed copy
  }

  tc::fence_before_sync();
  __syncthreads();
  // after a timeout, the products issued last complete before TMEM is freed (bounded)
  if (err && g > 0 && tid == 0) tc::mbar_wait(&full[(g - 1) & 1], ((g - 1) >> 1) & 1, kWaitCycles);
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
  if (tid == 0 && err && status) atomicCAS(&status->code, 0, (int)TKS_ETIMEOUT);
}

}  // namespace

size_t sketch3_smem_bytes(const int r[3]) {
  const size_t core = ((size_t)r[0] * r[1] * r[2] * 2 + 15) & ~(size_t)15;
  // the transposed copies have rows of r_n | 1 elements
  size_t copy = 0;
  for (int n = 1; n < 3; ++n) {
    const size_t c = (size_t)(r[n] | 1) * (n == 1 ? r[0] * r[2] : r[0] * r[1]) * 2;
    copy = c > copy ? c : copy;
  }
  copy = (copy + 15) & ~(size_t)15;
  return (size_t)kGOff + core + (copy > (size_t)kRedBytes ? copy : (size_t)kRedBytes);
}

bool sketch3_two_per_sm(const int r[3]) { return sketch3_smem_bytes(r) <= 112 * 1024; }

cudaError_t prepare_sketch3() {
  const int r[3] = {kMaxR, kMaxR, kMaxR};
  return cudaFuncSetAttribute(sketch3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sketch3_smem_bytes(r));
}

void launch_sketch3(const Sketch3Job* jobs, int njobs, size_t smem, const Bases& bases, Status* status,
                    cudaStream_t stream) {
  sketch3_tc_kernel<<<njobs, kThreads, smem, stream>>>(jobs, bases, status);
}

}  // namespace tks

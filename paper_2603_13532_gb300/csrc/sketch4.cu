// Khatri-Rao core sketches of an order-4 term, all four modes in one CTA (mixed-precision path).
//
// Alg. 4 (KRPSum-Tucker), Sec. 3.1.1: with M_m = U_k^(m)T Omega_m (r_m x s), column c of the mode-n
// sketch is V_kn[i_n, c] = sum over the other indices of G_k[i0, i1, i2, i3] prod_{j != n} M_j[i_j, c].
// Per column c, one pass over the core gives all four:
//   z[i0, i1, i2]  = sum_i3 G[i0, i1, i2, i3] M_3[i3, c]
//   w[i0, i1]      = sum_i2 z M_2[i2, c]
//   V_0[i0] += w M_1[i1],   V_1[i1] += w M_0[i0],   V_2[i2] += z M_0[i0] M_1[i1],
//   V_3[i3] += G[i0, i1, i2, i3] M_0[i0] M_1[i1] M_2[i2]
// (2 r^4 s multiply-adds per term instead of 4 r^4 s for four separate contractions).  Thread
// (group g, column c): c < s <= 64 owns one sketch column, the four groups split i1; the core is
// staged in shared memory as bf16 in slices of kc mode-1 indices, i3 fastest (8-byte loads of four
// values), and M_3's column and the V_3 partial sums live in registers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "bf16.cuh"
#include "kernels.h"

namespace tks {

namespace {

constexpr int kCols = 64;                  // sketch columns per CTA (s <= 64)
constexpr int kGroups = 4;                 // thread groups splitting i1
constexpr int kMaxR = kSketch4MaxRank;     // 24
constexpr int kQ3 = kMaxR / 4;             // quads of i3
constexpr int kThreads = kCols * kGroups;

__device__ __forceinline__ float lo_bf16(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_bf16(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ void store_planes(const Bases& bases, const Operand* planes, int64_t off, float v) {
  uint16_t h0, h1, h2;
  split3(v, h0, h1, h2);
  at<uint16_t>(bases, planes[0])[off] = h0;
  at<uint16_t>(bases, planes[1])[off] = h1;
  at<uint16_t>(bases, planes[2])[off] = h2;
}

__global__ void __launch_bounds__(kThreads) sketch4_term_kernel(const Sketch4Job* __restrict__ jobs, Bases bases) {
  extern __shared__ __align__(16) float s4s[];
  const Sketch4Job& J = jobs[blockIdx.x];
  const int r0 = J.r[0], r1 = J.r[1], r2 = J.r[2], r3 = J.r[3], s = J.s, kc = J.kc;
  const int r3p = (r3 + 3) & ~3;
  const int tid = threadIdx.x, c = tid % kCols, grp = tid / kCols;
  const bool live = c < s;
  float* M0s = s4s;                                   // [i0][c]
  float* M1s = M0s + kMaxR * kCols;                   // [i1][c]
  float* M2s = M1s + kMaxR * kCols;                   // [i2][c]
  float* V1s = M2s + kMaxR * kCols;                   // [i1][c], complete sums (i1 belongs to one group)
  float* V0p = V1s + kMaxR * kCols;                   // [grp][i0][c] partial sums (later V_3 partials)
  float* V2p = V0p + kGroups * kMaxR * kCols;         // [grp][i2][c] partial sums
  uint16_t* Gs = reinterpret_cast<uint16_t*>(V2p + kGroups * kMaxR * kCols);   // [i0l][i1][i2][i3p]
  const uint16_t* G = at<uint16_t>(bases, J.core);
  const float* Mg[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) Mg[m] = at<float>(bases, J.M[m]) + J.roff[m];

  float* Ms[3] = {M0s, M1s, M2s};
#pragma unroll
  for (int m = 0; m < 3; ++m)
    for (int e = tid; e < J.r[m] * kCols; e += kThreads) {
      const int i = e % J.r[m], cc = e / J.r[m];
      Ms[m][i * kCols + cc] = cc < s ? Mg[m][i + (int64_t)J.R[m] * cc] : 0.f;
    }
  for (int e = tid; e < kMaxR * kCols; e += kThreads) V1s[e] = 0.f;
  for (int e = tid; e < kGroups * kMaxR * kCols; e += kThreads) {
    V0p[e] = 0.f;
    V2p[e] = 0.f;
  }
  float m3[kMaxR], v3[kMaxR];
#pragma unroll
  for (int i = 0; i < kMaxR; ++i) {
    m3[i] = (i < r3 && live) ? Mg[3][i + (int64_t)J.R[3] * c] : 0.f;
    v3[i] = 0.f;
  }
  if (r3p > r3) {   // the padding i3 in [r3, r3p) of every row stays zero
    const int rows = kc * r1 * r2;
    for (int e = tid; e < rows * (r3p - r3); e += kThreads) Gs[(e / (r3p - r3)) * r3p + r3 + e % (r3p - r3)] = 0;
  }
  for (int a0 = 0; a0 < r0; a0 += kc) {
    const int nc = min(kc, r0 - a0);
    __syncthreads();   // the previous slice is no longer read
    // slice G[a0 .. a0 + nc)[:, :, :] into Gs[((i0 - a0) r1 + i1) r2 + i2][i3]; the walk follows the
    // core's own order (i0 fastest) so that neighbouring threads read neighbouring elements
    const int tot = nc * r1 * r2 * r3;
    for (int e = tid; e < tot; e += kThreads) {
      const int i0l = e % nc, rest = e / nc;   // rest = i1 + r1 (i2 + r2 i3)
      const int i1 = rest % r1, rest2 = rest / r1;
      const int i2 = rest2 % r2, i3 = rest2 / r2;
      Gs[((i0l * r1 + i1) * r2 + i2) * r3p + i3] = G[(a0 + i0l) + (int64_t)r0 * rest];
    }
    __syncthreads();
    for (int i1 = grp; i1 < r1; i1 += kGroups) {
      const float m1 = M1s[i1 * kCols + c];
      float v1 = 0.f;
      for (int i0l = 0; i0l < nc; ++i0l) {
        const int i0 = a0 + i0l;
        const float m0 = M0s[i0 * kCols + c];
        const float p01 = m0 * m1;
        float w = 0.f;
        const uint16_t* row = Gs + (size_t)(i0l * r1 + i1) * r2 * r3p;
        for (int i2 = 0; i2 < r2; ++i2) {
          const float m2 = M2s[i2 * kCols + c];
          const float p012 = p01 * m2;
          float za = 0.f, zb = 0.f;
#pragma unroll
          for (int q = 0; q < kQ3; ++q) {
            if (4 * q >= r3) continue;
            const uint2 pk = *reinterpret_cast<const uint2*>(row + i2 * r3p + 4 * q);
            const float g0 = lo_bf16(pk.x), g1 = hi_bf16(pk.x), g2 = lo_bf16(pk.y), g3 = hi_bf16(pk.y);
            za = fmaf(g0, m3[4 * q], za);
            zb = fmaf(g1, m3[4 * q + 1], zb);
            za = fmaf(g2, m3[4 * q + 2], za);
            zb = fmaf(g3, m3[4 * q + 3], zb);
            v3[4 * q] = fmaf(g0, p012, v3[4 * q]);
            v3[4 * q + 1] = fmaf(g1, p012, v3[4 * q + 1]);
            v3[4 * q + 2] = fmaf(g2, p012, v3[4 * q + 2]);
            v3[4 * q + 3] = fmaf(g3, p012, v3[4 * q + 3]);
          }
          const float z = za + zb;
          w = fmaf(z, m2, w);
          V2p[(grp * kMaxR + i2) * kCols + c] = fmaf(z, p01, V2p[(grp * kMaxR + i2) * kCols + c]);
        }
        V0p[(grp * kMaxR + i0) * kCols + c] = fmaf(w, m1, V0p[(grp * kMaxR + i0) * kCols + c]);
        v1 = fmaf(w, m0, v1);
      }
      V1s[i1 * kCols + c] += v1;
    }
  }
  __syncthreads();
  // V_1 (complete), V_0 and V_2 (sums over the groups)
  for (int e = tid; e < r1 * kCols; e += kThreads) {
    const int i = e % r1, cc = e / r1;
    if (cc < s) store_planes(bases, J.V[1], (J.roff[1] + i) + (int64_t)J.ldv[1] * cc, J.alpha * V1s[i * kCols + cc]);
  }
  for (int e = tid; e < r0 * kCols; e += kThreads) {
    const int i = e % r0, cc = e / r0;
    if (cc < s) {
      float v = 0.f;
#pragma unroll
      for (int g = 0; g < kGroups; ++g) v += V0p[(g * kMaxR + i) * kCols + cc];
      store_planes(bases, J.V[0], (J.roff[0] + i) + (int64_t)J.ldv[0] * cc, J.alpha * v);
    }
  }
  for (int e = tid; e < r2 * kCols; e += kThreads) {
    const int i = e % r2, cc = e / r2;
    if (cc < s) {
      float v = 0.f;
#pragma unroll
      for (int g = 0; g < kGroups; ++g) v += V2p[(g * kMaxR + i) * kCols + cc];
      store_planes(bases, J.V[2], (J.roff[2] + i) + (int64_t)J.ldv[2] * cc, J.alpha * v);
    }
  }
  __syncthreads();   // V0p is free: it takes the V_3 partial sums
#pragma unroll
  for (int i = 0; i < kMaxR; ++i)
    if (i < r3) V0p[(grp * kMaxR + i) * kCols + c] = v3[i];
  __syncthreads();
  for (int e = tid; e < r3 * kCols; e += kThreads) {
    const int i = e % r3, cc = e / r3;
    if (cc < s) {
      float v = 0.f;
#pragma unroll
      for (int g = 0; g < kGroups; ++g) v += V0p[(g * kMaxR + i) * kCols + cc];
      store_planes(bases, J.V[3], (J.roff[3] + i) + (int64_t)J.ldv[3] * cc, J.alpha * v);
    }
  }
}

constexpr size_t kFixedFloats = (size_t)(4 + 2 * kGroups) * kMaxR * kCols;

}  // namespace

int sketch4_slice(const int r[4], size_t budget_bytes) {
  const size_t slab = (size_t)2 * r[1] * r[2] * ((r[3] + 3) & ~3);
  const int kc = (int)std::max<size_t>(1, budget_bytes / slab);
  return kc < r[0] ? kc : r[0];
}

size_t sketch4_smem_bytes(const int r[4], int kc) {
  return sizeof(float) * kFixedFloats + (size_t)2 * kc * r[1] * r[2] * ((r[3] + 3) & ~3);
}

cudaError_t prepare_sketch4() {
  return cudaFuncSetAttribute(sketch4_term_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void launch_sketch4(const Sketch4Job* jobs, int njobs, size_t smem, const Bases& bases, cudaStream_t stream) {
  sketch4_term_kernel<<<njobs, kThreads, smem, stream>>>(jobs, bases);
}

}  // namespace tks

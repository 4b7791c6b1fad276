// Khatri-Rao core sketches of an order-3 term, all three modes in one CTA (mixed-precision path).
//
// Alg. 4 (KRPSum-Tucker), Sec. 3.1.1: with M_m = U_k^(m)T Omega_m (r_m x s) the sketch of mode n
// is V_kn = G_k,(n) (M_j2 (.) M_j1) (r_n x s), i.e. column c is G_k contracted with column c of
// the two other M's.  One CTA per term loads the core once and forms
//   Z[i0, i1, c]  = sum_i2 G[i0, i1, i2] M_2[i2, c]
//   V_0[i0, c]    = sum_i1 Z[i0, i1, c] M_1[i1, c]          V_1[i1, c] = sum_i0 Z[i0, i1, c] M_0[i0, c]
//   V_2[i2, c]    = sum_i1 M_1[i1, c] sum_i0 G[i0, i1, i2] M_0[i0, c]
// so modes 0 and 1 share the contraction over i2 (4 r0 r1 r2 s flops per term instead of 6).
// Thread (group g, column c): c < s <= 64 owns one sketch column; the four groups split i1 (first
// pass) and i2 (second pass).  Contractions run along the contiguous index of a zero-padded copy
// of the core in shared memory (i2 fastest for the first pass, i0 fastest for the second), four
// bf16 values per 8-byte load, against the thread's column of M_2 or M_0 held in registers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bf16.cuh"
#include "fastdiv.cuh"
#include "kernels.h"

namespace tks {

namespace {

constexpr int kCols = 64;       // sketch columns per CTA (s <= 64)
constexpr int kGroups = 4;      // thread groups splitting i1 / i2
constexpr int kMaxR = kSketch3MaxRank;
constexpr int kQuads = kMaxR / 4;
constexpr int kThreads = kCols * kGroups;
constexpr int kBatch = 8;       // core elements loaded per thread before they are stored

__device__ __forceinline__ float lo_bf16(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float hi_bf16(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// four consecutive core values starting at a 4-aligned index
__device__ __forceinline__ float4 load4(const uint16_t* p) {
  const uint2 pk = *reinterpret_cast<const uint2*>(p);
  return make_float4(lo_bf16(pk.x), hi_bf16(pk.x), lo_bf16(pk.y), hi_bf16(pk.y));
}
__device__ __forceinline__ float4 load4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ uint16_t to_core(uint16_t h, uint16_t) { return h; }
__device__ __forceinline__ float to_core(uint16_t h, float) { return __uint_as_float((uint32_t)h << 16); }

constexpr size_t kF32Smem = 110 * 1024;   // largest float32-core CTA (two per SM)

size_t smem_for(int r0, int r1, int r2, int r2p, bool f32) {
  const size_t r0p = (r0 + 3) & ~3;
  const size_t g = (size_t)r2p * r0 * r1 > r0p * r1 * r2 ? (size_t)r2p * r0 * r1 : r0p * r1 * r2;
  return sizeof(float) * (2 + kGroups) * kMaxR * kCols + (f32 ? 4 : 2) * g;
}

// Row stride of the first-pass core copy (i2 fastest): a multiple of 4 for the 16-byte reads.
// Float32 copies take 4 mod 8 where that still fits two CTAs per SM, so that the staging stores
// of consecutive i0 (r2p floats apart) are 4-way bank conflicts instead of up to 32-way (r2p = 32);
// the bf16 launch keeps the plain stride (its shared memory is that of its largest term).
int pass1_stride(int r0, int r1, int r2, bool f32) {
  const int p = (r2 + 3) & ~3;
  if (!f32 || (p & 7) != 0) return p;
  return smem_for(r0, r1, r2, p + 4, true) <= kF32Smem ? p + 4 : p;
}

__device__ __forceinline__ void store_planes(const Bases& bases, const Operand* planes, int64_t off, float v) {
  uint16_t h0, h1, h2;
  split3(v, h0, h1, h2);
  at<uint16_t>(bases, planes[0])[off] = h0;
  at<uint16_t>(bases, planes[1])[off] = h1;
  at<uint16_t>(bases, planes[2])[off] = h2;
}

// CoreT: the element type of the core copies in shared memory (float: converted once while
// staging, so the contractions load 16 bytes per four values; bf16: half the shared memory).
template <typename CoreT>
__global__ void __launch_bounds__(kThreads) sketch3_term_kernel(const Sketch3Job* __restrict__ jobs, Bases bases) {
  extern __shared__ __align__(16) float s3s[];
  const Sketch3Job& J = jobs[blockIdx.x];
  const int r0 = J.r[0], r1 = J.r[1], r2 = J.r[2], s = J.s;
  const int r0p = (r0 + 3) & ~3, r2p = J.r2p;
  const int tid = threadIdx.x, c = tid % kCols, grp = tid / kCols;
  const bool live = c < s;
  float* M0s = s3s;                                   // [i0][c]
  float* M1s = M0s + kMaxR * kCols;                   // [i1][c]
  float* V0p = M1s + kMaxR * kCols;                   // [grp][i0][c], partial sums of V_0
  CoreT* Gb = reinterpret_cast<CoreT*>(V0p + kGroups * kMaxR * kCols);
  const uint16_t* G = at<uint16_t>(bases, J.core);
  const float* Mg0 = at<float>(bases, J.M[0]) + J.roff[0];
  const float* Mg1 = at<float>(bases, J.M[1]) + J.roff[1];
  const float* Mg2 = at<float>(bases, J.M[2]) + J.roff[2];
  const int tot = r0 * r1 * r2;   // <= 2^15: the index quotients below are SmallDiv's
  const SmallDiv dr0(r0), dr1(r1);

  for (int e = tid; e < r0 * kCols; e += kThreads) {
    const int cc = dr0.quo(e), i = e - cc * r0;
    M0s[i * kCols + cc] = cc < s ? Mg0[i + (int64_t)J.R[0] * cc] : 0.f;
  }
  for (int e = tid; e < r1 * kCols; e += kThreads) {
    const int cc = dr1.quo(e), i = e - cc * r1;
    M1s[i * kCols + cc] = cc < s ? Mg1[i + (int64_t)J.R[1] * cc] : 0.f;
  }
  // first-pass copy of the core: Gb[i2 + r2p (i0 + r0 i1)], zero for i2 in [r2, r2p)
  if (r2p > r2) {
    const SmallDiv dp(r2p - r2);
    for (int e = tid; e < r0 * r1 * (r2p - r2); e += kThreads) {
      const int rest = dp.quo(e), pad = e - rest * (r2p - r2);
      Gb[r2 + pad + r2p * rest] = CoreT(0);
    }
  }
  for (int e0 = 0; e0 < tot; e0 += kBatch * kThreads) {
    // kBatch independent loads in flight per thread before the scattered shared-memory stores
    uint16_t v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * kThreads + tid;
      v[u] = e < tot ? G[e] : 0;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * kThreads + tid;
      if (e < tot) {
        const int q = dr0.quo(e), i0 = e - q * r0, i2 = dr1.quo(q), i1 = q - i2 * r1;
        Gb[i2 + r2p * (i0 + r0 * i1)] = to_core(v[u], CoreT());
      }
    }
  }
  float m2[kMaxR];
#pragma unroll
  for (int i = 0; i < kMaxR; ++i) m2[i] = (i < r2 && live) ? Mg2[i + (int64_t)J.R[2] * c] : 0.f;
  __syncthreads();

  // pass 1: modes 0 and 1
  float v0[kMaxR];
#pragma unroll
  for (int i = 0; i < kMaxR; ++i) v0[i] = 0.f;
  for (int i1 = grp; i1 < r1; i1 += kGroups) {
    const float m1 = M1s[i1 * kCols + c];
    float v1 = 0.f;
#pragma unroll
    for (int q0 = 0; q0 < kQuads; ++q0) {
      if (4 * q0 >= r0) continue;
      float z[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q2 = 0; q2 < kQuads; ++q2) {
        if (4 * q2 >= r2) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // rows i0 >= r0 of the last quad read the next core fibre (or the padding); their z is unused
          const int i0 = min(4 * q0 + j, r0 - 1);
          const float4 gv = load4(Gb + r2p * (i0 + r0 * i1) + 4 * q2);
          z[j] = fmaf(gv.x, m2[4 * q2], z[j]);
          z[j] = fmaf(gv.y, m2[4 * q2 + 1], z[j]);
          z[j] = fmaf(gv.z, m2[4 * q2 + 2], z[j]);
          z[j] = fmaf(gv.w, m2[4 * q2 + 3], z[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i0 = 4 * q0 + j;
        if (i0 < r0) {
          v0[i0] = fmaf(z[j], m1, v0[i0]);
          v1 = fmaf(z[j], M0s[i0 * kCols + c], v1);
        }
      }
    }
    if (live) store_planes(bases, J.V[1], (J.roff[1] + i1) + (int64_t)J.ldv[1] * c, J.alpha * v1);
  }
#pragma unroll
  for (int i = 0; i < kMaxR; ++i)
    if (i < r0) V0p[(grp * kMaxR + i) * kCols + c] = v0[i];
  __syncthreads();   // pass 1 is done with Gb; the V_0 partials are in place
  for (int e = tid; e < r0 * kCols; e += kThreads) {
    const int cc = dr0.quo(e), i = e - cc * r0;   // runs of consecutive rows of one column
    if (cc < s) {
      float v = 0.f;
#pragma unroll
      for (int g = 0; g < kGroups; ++g) v += V0p[(g * kMaxR + i) * kCols + cc];
      store_planes(bases, J.V[0], (J.roff[0] + i) + (int64_t)J.ldv[0] * cc, J.alpha * v);
    }
  }
  // second-pass copy: Gb[i0 + r0p (i1 + r1 i2)], zero for i0 in [r0, r0p)
  if (r0p > r0) {
    const SmallDiv dp(r0p - r0);
    for (int e = tid; e < r1 * r2 * (r0p - r0); e += kThreads) {
      const int rest = dp.quo(e), pad = e - rest * (r0p - r0);
      Gb[r0 + pad + r0p * rest] = CoreT(0);
    }
  }
  for (int e0 = 0; e0 < tot; e0 += kBatch * kThreads) {
    uint16_t v[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * kThreads + tid;
      v[u] = e < tot ? G[e] : 0;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * kThreads + tid;
      if (e < tot) {
        const int q = dr0.quo(e);
        Gb[e - q * r0 + r0p * q] = to_core(v[u], CoreT());
      }
    }
  }
  float m0[kMaxR];
#pragma unroll
  for (int i = 0; i < kMaxR; ++i) m0[i] = (i < r0) ? M0s[i * kCols + c] : 0.f;
  __syncthreads();

  // pass 2: mode 2
  for (int i2 = grp; i2 < r2; i2 += kGroups) {
    float acc = 0.f;
    for (int i1 = 0; i1 < r1; ++i1) {
      const CoreT* g = Gb + r0p * (i1 + r1 * i2);
      float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q0 = 0; q0 < kQuads; ++q0) {
        if (4 * q0 >= r0) continue;
        const float4 gv = load4(g + 4 * q0);
        y[0] = fmaf(gv.x, m0[4 * q0], y[0]);
        y[1] = fmaf(gv.y, m0[4 * q0 + 1], y[1]);
        y[2] = fmaf(gv.z, m0[4 * q0 + 2], y[2]);
        y[3] = fmaf(gv.w, m0[4 * q0 + 3], y[3]);
      }
      acc = fmaf((y[0] + y[1]) + (y[2] + y[3]), M1s[i1 * kCols + c], acc);
    }
    if (live) store_planes(bases, J.V[2], (J.roff[2] + i2) + (int64_t)J.ldv[2] * c, J.alpha * acc);
  }
}

}  // namespace

size_t sketch3_smem_bytes(const int r[3], bool f32_core) {
  return smem_for(r[0], r[1], r[2], pass1_stride(r[0], r[1], r[2], f32_core), f32_core);
}

int sketch3_stride(const int r[3], bool f32_core) { return pass1_stride(r[0], r[1], r[2], f32_core); }

bool sketch3_fits_f32(const int r[3]) { return smem_for(r[0], r[1], r[2], (r[2] + 3) & ~3, true) <= kF32Smem; }

cudaError_t prepare_sketch3() {
  cudaError_t e =
      cudaFuncSetAttribute(sketch3_term_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(sketch3_term_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void launch_sketch3(const Sketch3Job* jobs, int njobs, size_t smem, bool f32_core, const Bases& bases,
                    cudaStream_t stream) {
  if (f32_core)
    sketch3_term_kernel<float><<<njobs, kThreads, smem, stream>>>(jobs, bases);
  else
    sketch3_term_kernel<uint16_t><<<njobs, kThreads, smem, stream>>>(jobs, bases);
}

}  // namespace tks

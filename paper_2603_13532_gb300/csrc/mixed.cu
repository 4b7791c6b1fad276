// Float32 CUDA-core kernels of the mixed-precision path: the small ragged contractions
// (per-term core chains, core sketch), conversion of float64 bases into bfloat16 planes and
// the transpose of the concatenated factors into the K-major layout the tensor-core GEMMs read.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bf16.cuh"
#include "kernels.h"

namespace tks {

namespace {

template <typename Job>
__device__ __forceinline__ int find_begin(const Job* jobs, int njobs, int64_t key) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].begin <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float load_typed(const char* base, int32_t type, int64_t idx) {
  switch (type) {
    case T_F64: return (float)reinterpret_cast<const double*>(base)[idx];
    case T_F32: return reinterpret_cast<const float*>(base)[idx];
    default: return bf16_float(reinterpret_cast<const uint16_t*>(base)[idx]);
  }
}

// ----------------------------------------------------------------------------- SIMT GEMM
constexpr int ST = 64, SK = 16;

__global__ void __launch_bounds__(256) simt_gemm_f32_kernel(const SimtJob* __restrict__ jobs, int njobs,
                                                            Bases bases) {
  __shared__ float As[SK][ST + 1];
  __shared__ float Bs[SK][ST + 1];
  const int lo = tile_job(jobs, njobs, (int)blockIdx.x);
  const SimtJob& J = jobs[lo];
  int local = blockIdx.x - J.tile_begin;
  const int tn = local % J.tiles_n;
  local /= J.tiles_n;
  const int tm = local % J.tiles_m;
  const int bt = local / J.tiles_m;
  const char* A = at<char>(bases, J.A);
  const char* B = at<char>(bases, J.B);
  const int64_t a_bt = bt * J.a_b, b_bt = bt * J.b_b;
  const int m0 = tm * ST, n0 = tn * ST;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool a_mfast = (J.a_m == 1), b_kfast = (J.b_k0 == 1);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < J.K; k0 += SK) {
    for (int e = threadIdx.x; e < ST * SK; e += 256) {
      int i, kk;
      if (a_mfast) { i = e % ST; kk = e / ST; } else { kk = e % SK; i = e / SK; }
      const int gi = m0 + i, gk = k0 + kk;
      float v = 0.f;
      if (gi < J.M && gk < J.K) {
        const int kq = gk / J.K1, kr = gk - kq * J.K1;
        v = load_typed(A, J.a_type, a_bt + gi * J.a_m + kr * J.a_k0 + kq * J.a_k1);
      }
      As[kk][i] = v;
      int jj;
      if (b_kfast) { kk = e % SK; jj = e / SK; } else { jj = e % ST; kk = e / ST; }
      const int gj = n0 + jj, gk2 = k0 + kk;
      float w = 0.f;
      if (gj < J.N && gk2 < J.K) {
        const int kq = gk2 / J.K1, kr = gk2 - kq * J.K1;
        w = load_typed(B, J.b_type, b_bt + gj * J.b_n + kr * J.b_k0 + kq * J.b_k1);
      }
      Bs[kk][jj] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* c32 = J.has_c32 ? at<float>(bases, J.c32) : nullptr;
  double* c64 = J.has_c64 ? at<double>(bases, J.c64) : nullptr;
  uint16_t* cb0 = J.nbf > 0 ? at<uint16_t>(bases, J.cb[0]) : nullptr;
  uint16_t* cb1 = J.nbf > 1 ? at<uint16_t>(bases, J.cb[1]) : nullptr;
  uint16_t* cb2 = J.nbf > 2 ? at<uint16_t>(bases, J.cb[2]) : nullptr;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
      if (gi < J.M && gj < J.N) {
        const int64_t off = bt * J.c_b + gi * J.c_m + gj * J.c_n;
        const float v = J.alpha * acc[i][j];
        if (c32) c32[off] = v;
        if (c64) c64[off] = f32_to_f64_exact(v);
        if (cb0) {
          uint16_t h0, h1, h2;
          split3(v, h0, h1, h2);
          cb0[off] = h0;
          if (cb1) cb1[off] = h1;
          if (cb2) cb2[off] = h2;
        }
      }
    }
}

// ----------------------------------------------------------------------------- core sketch
// Same contraction as the float64 kernel (Eqs. krp_sketch_result / kron_sketch_result) with a
// bfloat16 core, float32 sketched factors M_j and float32 accumulation.
__global__ void core_sketch_f32_kernel(const CoreSketchF32Job* __restrict__ jobs, int njobs, int64_t total,
                                       Bases bases) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const CoreSketchF32Job& J = jobs[find_begin(jobs, njobs, g)];
    const int64_t e = g - J.begin;
    const int d = J.d, n = J.n;
    const int a = (int)(e % J.r[n]);
    const int c = (int)(e / J.r[n]);
    int col[MAXD], others[MAXD], st[MAXD];
    int no = 0;
    {
      int rem = c, stride = 1;
      for (int j = 0; j < d; ++j) {
        st[j] = stride;
        stride *= J.r[j];
        if (j == n) continue;
        others[no++] = j;
        if (J.kron) { col[j] = rem % J.s[j]; rem /= J.s[j]; } else { col[j] = c; }
      }
    }
    const uint16_t* G = at<uint16_t>(bases, J.core);
    const float* Mcol[MAXD];
    for (int t = 0; t < no; ++t) {
      const int j = others[t];
      Mcol[t] = at<float>(bases, J.M[j]) + J.roff[j] + (int64_t)J.R[j] * col[j];
    }
    const int f = others[0];
    const int rf = J.r[f], sf = st[f];
    int idx[MAXD];
    for (int t = 0; t < no; ++t) idx[t] = 0;
    int64_t goff = (int64_t)a * st[n];
    float acc = 0.f;
    while (true) {
      float prod = 1.f;
      for (int t = 1; t < no; ++t) prod *= Mcol[t][idx[t]];
      float inner = 0.f;
      const float* mf = Mcol[0];
      for (int i = 0; i < rf; ++i) inner = fmaf(bf16_float(G[goff + (int64_t)i * sf]), mf[i], inner);
      acc = fmaf(prod, inner, acc);
      int t = 1;
      for (; t < no; ++t) {
        const int j = others[t];
        goff += st[j];
        if (++idx[t] < J.r[j]) break;
        goff -= (int64_t)st[j] * J.r[j];
        idx[t] = 0;
      }
      if (t >= no) break;
    }
    const int64_t off = (J.roff[n] + a) + (int64_t)J.ldv * c;
    uint16_t h0, h1, h2;
    split3(J.alpha * acc, h0, h1, h2);
    at<uint16_t>(bases, J.V[0])[off] = h0;
    at<uint16_t>(bases, J.V[1])[off] = h1;
    at<uint16_t>(bases, J.V[2])[off] = h2;
  }
}


// ----------------------------------------------------------------------------- order-3 kernels
// Khatri-Rao core sketch of one (term, mode n) of an order-3 problem, in shared memory:
//   V[a, c] = alpha sum_{p2} M2[p2, c] sum_{p1} G[a, p1, p2] M1[p1, c]
// (p1, p2 the rank indices of the two other modes in ascending order).  A thread owns one column
// c and 8 consecutive rows a: per (p1, p2) it loads one M1 value and the 8 core values as one
// 16-byte broadcast, so each shared-memory wavefront feeds several FMAs.  V is staged in shared
// memory and written with a fastest.
constexpr int kCsRows = 8;

__global__ void __launch_bounds__(256) core_sketch_krp3_kernel(const CoreSketchF32Job* __restrict__ jobs,
                                                               Bases bases) {
  extern __shared__ __align__(16) float sm3[];
  const CoreSketchF32Job& J = jobs[blockIdx.x];
  const int n = J.n;
  const int j1 = (n == 0) ? 1 : 0, j2 = (n == 2) ? 1 : 2;
  const int rn = J.r[n], r1 = J.r[j1], r2 = J.r[j2], s = J.S;
  const int rnp = (rn + kCsRows - 1) / kCsRows * kCsRows;   // rows padded to whole 8-row groups
  float* M1 = sm3;                       // [c + s p1]
  float* M2 = M1 + r1 * s;               // [c + s p2]
  float* Vs = M2 + r2 * s;               // [a + rnp c]
  // [a + rnp (p1 + r1 p2)], base rounded up to 16 bytes for the 8-wide loads
  uint16_t* Gs = reinterpret_cast<uint16_t*>((reinterpret_cast<uintptr_t>(Vs + rnp * s) + 15) & ~uintptr_t(15));
  const uint16_t* G = at<uint16_t>(bases, J.core);
  const int tot = rn * r1 * r2;
  {
    int dst_stride[3];
    dst_stride[n] = 1;
    dst_stride[j1] = rnp;
    dst_stride[j2] = rnp * r1;
    const int q0 = J.r[0], q1 = J.r[1];
    for (int e = threadIdx.x; e < rnp * r1 * r2; e += blockDim.x) Gs[e] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int i0 = e % q0, i1 = (e / q0) % q1, i2 = e / (q0 * q1);
      Gs[i0 * dst_stride[0] + i1 * dst_stride[1] + i2 * dst_stride[2]] = G[e];
    }
  }
  const float* Mg1 = at<float>(bases, J.M[j1]) + J.roff[j1];
  const float* Mg2 = at<float>(bases, J.M[j2]) + J.roff[j2];
  for (int e = threadIdx.x; e < r1 * s; e += blockDim.x) {
    const int c = e % s, p = e / s;
    M1[e] = Mg1[p + (int64_t)J.R[j1] * c];
  }
  for (int e = threadIdx.x; e < r2 * s; e += blockDim.x) {
    const int c = e % s, p = e / s;
    M2[e] = Mg2[p + (int64_t)J.R[j2] * c];
  }
  __syncthreads();
  const int groups = rnp / kCsRows;
  for (int e = threadIdx.x; e < groups * s; e += blockDim.x) {
    const int c = e % s, a0 = (e / s) * kCsRows;
    float acc[kCsRows];
#pragma unroll
    for (int t = 0; t < kCsRows; ++t) acc[t] = 0.f;
    for (int p2 = 0; p2 < r2; ++p2) {
      float inner[kCsRows];
#pragma unroll
      for (int t = 0; t < kCsRows; ++t) inner[t] = 0.f;
      const uint16_t* g = Gs + a0 + rnp * r1 * p2;
      for (int p1 = 0; p1 < r1; ++p1) {
        const float m1 = M1[c + s * p1];
        const uint4 packed = *reinterpret_cast<const uint4*>(g + rnp * p1);
        const uint32_t w[4] = {packed.x, packed.y, packed.z, packed.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          inner[2 * t] = fmaf(__uint_as_float(w[t] << 16), m1, inner[2 * t]);
          inner[2 * t + 1] = fmaf(__uint_as_float(w[t] & 0xffff0000u), m1, inner[2 * t + 1]);
        }
      }
      const float m2 = M2[c + s * p2];
#pragma unroll
      for (int t = 0; t < kCsRows; ++t) acc[t] = fmaf(m2, inner[t], acc[t]);
    }
#pragma unroll
    for (int t = 0; t < kCsRows; ++t) Vs[a0 + t + rnp * c] = J.alpha * acc[t];
  }
  __syncthreads();
  uint16_t* V0 = at<uint16_t>(bases, J.V[0]);
  uint16_t* V1 = at<uint16_t>(bases, J.V[1]);
  uint16_t* V2 = at<uint16_t>(bases, J.V[2]);
  for (int e = threadIdx.x; e < rn * s; e += blockDim.x) {
    const int a = e % rn, c = e / rn;
    const int64_t off = (J.roff[n] + a) + (int64_t)J.ldv * c;
    uint16_t h0, h1, h2;
    split3(Vs[a + rnp * c], h0, h1, h2);
    V0[off] = h0;
    V1[off] = h1;
    V2[off] = h2;
  }
}

// Stage (c2) chain of one term of an order-3 problem for a block of AB <= 8 mode-1 rows, in shared
// memory:  W[ia, i1, c] = sum_{i0} A1[a0 + ia, i0] G[i0, i1, c]  (a thread owns one (c, i1) and all
// rows ia), then  T[ia, a1, c] = sum_{i1} W[ia, i1, c] A2[a1, i1]  (a thread owns one c, 4 columns
// a1 and all rows ia: 32 accumulators).  Threads run with c fastest so the Tcat writes
// ((roff_2 + c) + ldT J) come out in runs.
constexpr int kChainCols = 4;

__global__ void __launch_bounds__(256) chain3_kernel(const Chain3Job* __restrict__ jobs, Bases bases) {
  extern __shared__ float sc3[];
  const Chain3Job& J = jobs[blockIdx.x];
  const int r0 = J.r[0], r1 = J.r[1], r2 = J.r[2], b0 = J.b[0], b1 = J.b[1], AB = J.rows;
  constexpr int kAB = 8;
  float* A1 = sc3;                  // [ia + 8 i0]
  float* A2 = A1 + kAB * r0;        // [i1 + r1 a1]
  float* Ws = A2 + r1 * b1;         // [c + r2 (ia + 8 i1)]
  uint16_t* Gt = reinterpret_cast<uint16_t*>(Ws + r2 * kAB * r1);   // [c + r2 (i0 + r0 i1)]
  const uint16_t* G = at<uint16_t>(bases, J.core);
  for (int e = threadIdx.x; e < r0 * r1 * r2; e += blockDim.x) {
    const int i0 = e % r0, i1 = (e / r0) % r1, c = e / (r0 * r1);
    Gt[c + r2 * (i0 + r0 * i1)] = G[e];
  }
  const float* At1 = at<float>(bases, J.AT[0]) + J.roff[0];
  const float* At2 = at<float>(bases, J.AT[1]) + J.roff[1];
  for (int e = threadIdx.x; e < kAB * r0; e += blockDim.x) {
    const int ia = e % kAB, i0 = e / kAB;
    A1[e] = ia < AB ? At1[i0 + (int64_t)J.R[0] * (J.a0 + ia)] : 0.f;
  }
  for (int e = threadIdx.x; e < r1 * b1; e += blockDim.x) {
    const int i1 = e % r1, a1 = e / r1;
    A2[e] = At2[i1 + (int64_t)J.R[1] * a1];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r2 * r1; e += blockDim.x) {
    const int c = e % r2, i1 = e / r2;
    const uint16_t* g = Gt + c + r2 * r0 * i1;
    float w[kAB];
#pragma unroll
    for (int t = 0; t < kAB; ++t) w[t] = 0.f;
    for (int i0 = 0; i0 < r0; ++i0) {
      const float gv = bf16_float(g[r2 * i0]);
      const float4 a_lo = *reinterpret_cast<const float4*>(A1 + kAB * i0);
      const float4 a_hi = *reinterpret_cast<const float4*>(A1 + kAB * i0 + 4);
      w[0] = fmaf(a_lo.x, gv, w[0]);
      w[1] = fmaf(a_lo.y, gv, w[1]);
      w[2] = fmaf(a_lo.z, gv, w[2]);
      w[3] = fmaf(a_lo.w, gv, w[3]);
      w[4] = fmaf(a_hi.x, gv, w[4]);
      w[5] = fmaf(a_hi.y, gv, w[5]);
      w[6] = fmaf(a_hi.z, gv, w[6]);
      w[7] = fmaf(a_hi.w, gv, w[7]);
    }
#pragma unroll
    for (int t = 0; t < kAB; ++t) Ws[c + r2 * (t + kAB * i1)] = w[t];
  }
  __syncthreads();
  uint16_t* T0 = at<uint16_t>(bases, J.T[0]);
  uint16_t* T1 = at<uint16_t>(bases, J.T[1]);
  uint16_t* T2 = at<uint16_t>(bases, J.T[2]);
  const int ncol = (b1 + kChainCols - 1) / kChainCols;
  for (int e = threadIdx.x; e < r2 * ncol; e += blockDim.x) {
    const int c = e % r2, a1b = (e / r2) * kChainCols;
    float t[kAB][kChainCols];
#pragma unroll
    for (int x = 0; x < kAB; ++x)
#pragma unroll
      for (int y = 0; y < kChainCols; ++y) t[x][y] = 0.f;
    for (int i1 = 0; i1 < r1; ++i1) {
      float w[kAB], a2[kChainCols];
#pragma unroll
      for (int x = 0; x < kAB; ++x) w[x] = Ws[c + r2 * (x + kAB * i1)];
#pragma unroll
      for (int y = 0; y < kChainCols; ++y) a2[y] = (a1b + y < b1) ? A2[i1 + r1 * (a1b + y)] : 0.f;
#pragma unroll
      for (int x = 0; x < kAB; ++x)
#pragma unroll
        for (int y = 0; y < kChainCols; ++y) t[x][y] = fmaf(w[x], a2[y], t[x][y]);
    }
#pragma unroll
    for (int x = 0; x < kAB; ++x) {
      if (x >= AB) break;
#pragma unroll
      for (int y = 0; y < kChainCols; ++y) {
        const int a1 = a1b + y;
        if (a1 >= b1) break;
        const int64_t off = (J.roff[2] + c) + (int64_t)J.ldT * (J.a0 + x + (int64_t)b0 * a1);
        uint16_t h0, h1, h2;
        split3(J.alpha * t[x][y], h0, h1, h2);
        T0[off] = h0;
        T1[off] = h1;
        T2[off] = h2;
      }
    }
  }
}

// ----------------------------------------------------------------------------- split / transpose
// One CTA per tile of kSplitTile elements of one job (column-major element order): the tile's first
// element takes one 64-bit division, later ones step along the column.
__global__ void __launch_bounds__(256) split_f64_kernel(const SplitJob* __restrict__ jobs, int njobs, Bases bases) {
  const SplitJob& J = jobs[tile_job(jobs, njobs, (int)blockIdx.x)];
  const int64_t e0 = (int64_t)(blockIdx.x - J.tile_begin) * kSplitTile + threadIdx.x;
  int64_t j = e0 / J.rows, i = e0 - j * J.rows;
  const double* src = at<double>(bases, J.src);
  uint16_t* d0 = at<uint16_t>(bases, J.dst[0]);
  uint16_t* d1 = at<uint16_t>(bases, J.dst[1]);
  uint16_t* d2 = at<uint16_t>(bases, J.dst[2]);
#pragma unroll
  for (int k = 0; k < kSplitTile / 256; ++k) {
    if (e0 + 256 * k < J.count) {
      const double v = src[i + J.ld_src * j];
      uint16_t h0, h1, h2;
      split3(v, h0, h1, h2);
      const int64_t off = J.trans ? j + J.ld_dst * i : i + J.ld_dst * j;
      d0[off] = h0;
      d1[off] = h1;
      d2[off] = h2;
    }
    i += 256;
    while (i >= J.rows) {   // rows >= 1: at most 256 steps, one when rows >= 256
      i -= J.rows;
      ++j;
    }
  }
}

__global__ void __launch_bounds__(256) transpose_bf16_kernel(const TransposeJob* __restrict__ jobs, int njobs,
                                                             Bases bases) {
  // 64 x 64 tiles.  Full tiles with leading dimensions that are multiples of 8 move 16 bytes per
  // access: a column segment of 8 rows is read into row y of the shared tile (source order), the
  // tile's 16-byte chunks XOR-swizzled by y / 8 so that the reads of 8 column segments that feed one
  // 16-byte store of the destination hit distinct banks; each destination row gets 128 contiguous
  // bytes from 8 lanes.
  __shared__ __align__(16) uint16_t tile[64][66];
  const int lo = tile_job(jobs, njobs, (int)blockIdx.x);
  const TransposeJob& J = jobs[lo];
  const int local = blockIdx.x - J.tile_begin;
  const int tr = local % J.tiles_r, tcol = local / J.tiles_r;
  const uint16_t* src = at<uint16_t>(bases, J.src);
  uint16_t* dst = at<uint16_t>(bases, J.dst);
  const int i0 = tr * 64, j0 = tcol * 64;
  const bool vec = ((J.ld_src | J.ld_dst) & 7) == 0 && i0 + 64 <= J.rows && j0 + 64 <= J.cols;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 lanes x 8 warps
  if (vec) {
    uint4* t4 = reinterpret_cast<uint4*>(&tile[0][0]);       // viewed as [64 rows][8 chunks], no padding
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int idx = threadIdx.x + 256 * k;
      const int y = idx >> 3, seg = idx & 7;                // column j0 + y, rows i0 + 8 seg .. + 7
      const uint4 v = *reinterpret_cast<const uint4*>(src + (i0 + 8 * seg) + J.ld_src * (int64_t)(j0 + y));
      t4[y * 8 + (seg ^ ((y >> 3) & 7))] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int idx = threadIdx.x + 256 * k;
      const int jseg = idx & 7, i = idx >> 3;               // destination row i0 + i, columns j0 + 8 jseg .. + 7
      const uint16_t* tb = reinterpret_cast<const uint16_t*>(t4);
      uint32_t w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int y0 = 8 * jseg + 2 * u, y1 = y0 + 1;
        const uint32_t a = tb[(y0 * 8 + ((i >> 3) ^ jseg)) * 8 + (i & 7)];
        const uint32_t b = tb[(y1 * 8 + ((i >> 3) ^ jseg)) * 8 + (i & 7)];
        w[u] = a | (b << 16);
      }
      *reinterpret_cast<uint4*>(dst + (j0 + 8 * jseg) + J.ld_dst * (int64_t)(i0 + i)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  } else {
    for (int y = ty; y < 64; y += 8)
      for (int x = tx; x < 64; x += 32) {
        const int i = i0 + x, j = j0 + y;
        if (i < J.rows && j < J.cols) tile[x][y] = src[i + J.ld_src * (int64_t)j];
      }
    __syncthreads();
    for (int y = ty; y < 64; y += 8)
      for (int x = tx; x < 64; x += 32) {
        const int j = j0 + x, i = i0 + y;
        if (i < J.rows && j < J.cols) dst[j + J.ld_dst * (int64_t)i] = tile[y][x];
      }
  }
}

int grid_for(int64_t work, int threads) {
  const int64_t g = (work + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

}  // namespace

void launch_simt_gemm_f32(const SimtJob* jobs, int njobs, int total_tiles, const Bases& bases,
                          cudaStream_t stream) {
  simt_gemm_f32_kernel<<<total_tiles, 256, 0, stream>>>(jobs, njobs, bases);
}

void launch_core_sketch_f32(const CoreSketchF32Job* jobs, int njobs, int64_t total, const Bases& bases,
                            cudaStream_t stream) {
  core_sketch_f32_kernel<<<grid_for(total, 128), 128, 0, stream>>>(jobs, njobs, total, bases);
}

cudaError_t prepare_order3_kernels() {
  cudaError_t e = cudaFuncSetAttribute(core_sketch_krp3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       222 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(chain3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 222 * 1024);
}

void launch_core_sketch_krp3(const CoreSketchF32Job* jobs, int njobs, size_t smem, const Bases& bases,
                             cudaStream_t stream) {
  core_sketch_krp3_kernel<<<njobs, 256, smem, stream>>>(jobs, bases);
}

void launch_chain3(const Chain3Job* jobs, int njobs, size_t smem, const Bases& bases, cudaStream_t stream) {
  chain3_kernel<<<njobs, 256, smem, stream>>>(jobs, bases);
}

void launch_split_f64(const SplitJob* jobs, int njobs, int64_t tiles, const Bases& bases, cudaStream_t stream) {
  split_f64_kernel<<<(unsigned)tiles, 256, 0, stream>>>(jobs, njobs, bases);
}

void launch_transpose_bf16(const TransposeJob* jobs, int njobs, int total_tiles, const Bases& bases,
                           cudaStream_t stream) {
  transpose_bf16_kernel<<<total_tiles, 256, 0, stream>>>(jobs, njobs, bases);
}

}  // namespace tks

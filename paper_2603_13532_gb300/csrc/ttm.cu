// Mode products with a small matrix, float32 on the CUDA cores (mixed-precision ST-HOSVD).
//
// Alg. 2 phase 2 truncates the core mode by mode, H <- H x_n P_n^T, and the factors become
// U~_n = Q_n P_n.  Both are  Y[l, c, r] = sum_a X[l, a, r] P[a, c]  with X of shape (L, b, Rr)
// (l fastest) and P (b x rmax, rmax <= 64): a GEMM whose rows are the fibres q = (l, r).  A CTA
// takes 128 fibres: it stages them (b x 128) and P in shared memory with coalesced loads (along
// a when L = 1, along l otherwise), each thread forms an 8 x 4 register tile, and the 128 x rmax
// result goes back through shared memory so the stores are coalesced too.
#include <cuda_runtime.h>

#include "fastdiv.cuh"
#include "kernels.h"

namespace tks {

namespace {

constexpr int kRowsPerCta = 128;
constexpr int kThreads = 256;
constexpr int kMaxCols = 64;
constexpr int kBatch = 8;              // global loads in flight per thread while staging
constexpr int kXs = kRowsPerCta + 4;
static_assert(kThreads % kRowsPerCta == 0, "a thread keeps one fibre while staging along l");   // padded fibre-tile row (16-byte aligned, fewer bank conflicts)

__device__ __forceinline__ float load_elem(const char* base, int32_t type, int64_t idx) {
  return type == T_F64 ? (float)reinterpret_cast<const double*>(base)[idx] : reinterpret_cast<const float*>(base)[idx];
}

__global__ void __launch_bounds__(kThreads) ttm_rows_kernel(const TtmJob* __restrict__ jobs, int njobs, Bases bases) {
  extern __shared__ __align__(16) float tsm[];
  const int lo = tile_job(jobs, njobs, (int)blockIdx.x);
  const TtmJob& J = jobs[lo];
  const int b = J.b, rmax = J.rmax;
  const int64_t L = J.L, rows = J.L * J.Rr;
  const int64_t q0 = (int64_t)(blockIdx.x - J.tile_begin) * kRowsPerCta;
  const int64_t left = rows - q0;
  const int nq = left < kRowsPerCta ? (int)left : kRowsPerCta;
  float* Ps = tsm;                                   // [a][c], c < 64
  float* Xs = Ps + TKS_MAX_BASIS * kMaxCols;         // [a][q], row kXs (then [c][q] for the result)
  const char* X = at<char>(bases, J.X);
  const float* P = at<float>(bases, J.P);
  for (int e = threadIdx.x; e < b * kMaxCols; e += kThreads) {
    const int a = e / kMaxCols, c = e % kMaxCols;
    Ps[e] = c < rmax ? P[a + (int64_t)b * c] : 0.f;
  }
  // fibre q = l + L r starts at l + L b r; entry a at + L a
  // kBatch loads in flight per thread before the shared-memory stores
  if (L == 1) {
    // the tile's fibres are contiguous: elements e = q b + a of a run starting at q0 b
    const int total = b * kRowsPerCta, valid = b * nq;
    const SmallDiv db(b);
    for (int e0 = 0; e0 < total; e0 += kBatch * kThreads) {
      float v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int e = e0 + u * kThreads + threadIdx.x;
        v[u] = e < valid ? load_elem(X, J.x_type, q0 * b + e) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int e = e0 + u * kThreads + threadIdx.x;
        if (e < total) {   // e < TKS_MAX_BASIS kRowsPerCta < 2^16
          const int q = db.quo(e);
          Xs[(e - q * b) * kXs + q] = v[u];
        }
      }
    }
  } else {
    // a thread keeps one fibre q (kThreads is a multiple of kRowsPerCta) and steps through a
    constexpr int kStep = kThreads / kRowsPerCta;
    const int q = threadIdx.x % kRowsPerCta;
    int64_t base = 0;
    if (q < nq) {
      const int64_t g = q0 + q, r = g / L, l = g - r * L;
      base = l + L * (int64_t)b * r;
    }
    for (int a0 = threadIdx.x / kRowsPerCta; a0 < b; a0 += kBatch * kStep) {
      float v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int a = a0 + u * kStep;
        v[u] = (q < nq && a < b) ? load_elem(X, J.x_type, base + L * a) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int a = a0 + u * kStep;
        if (a < b) Xs[a * kXs + q] = v[u];
      }
    }
  }
  __syncthreads();
  const int tr = threadIdx.x % 16, tc = threadIdx.x / 16;   // rows 8 tr .. 8 tr + 7, cols 4 tc .. 4 tc + 3
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  // columns 4 tc .. 4 tc + 3 at or beyond rmax are never written out: their threads skip the
  // product (with rmax = 48 a quarter of the tile)
  const int bq = 4 * tc < rmax ? b : 0;
  for (int a = 0; a < bq; ++a) {
    const float4 x0 = *reinterpret_cast<const float4*>(Xs + a * kXs + 8 * tr);
    const float4 x1 = *reinterpret_cast<const float4*>(Xs + a * kXs + 8 * tr + 4);
    const float4 p = *reinterpret_cast<const float4*>(Ps + a * kMaxCols + 4 * tc);
    const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
    const float pv[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], pv[j], acc[i][j]);
  }
  __syncthreads();   // Xs is reused for the result [c][q]
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 8; ++i) Xs[(4 * tc + j) * kXs + 8 * tr + i] = acc[i][j];
  __syncthreads();
  // Y[l + L (c + rmax r)]: along c when L = 1, along l otherwise
  char* Y = at<char>(bases, J.Y);
  const bool f64 = J.y_type == T_F64;
  if (L == 1) {
    const SmallDiv dr(rmax);
    for (int e = threadIdx.x; e < rmax * nq; e += kThreads) {
      const int q = dr.quo(e), c = e - q * rmax;
      const int64_t off = c + (int64_t)rmax * (q0 + q);
      const float v = Xs[c * kXs + q];
      if (f64) reinterpret_cast<double*>(Y)[off] = (double)v; else reinterpret_cast<float*>(Y)[off] = v;
    }
  } else {
    const int q = threadIdx.x % kRowsPerCta;
    if (q < nq) {
      const int64_t g = q0 + q, r = g / L, l = g - r * L;
      const int64_t base = l + L * (int64_t)rmax * r;
      for (int c = threadIdx.x / kRowsPerCta; c < rmax; c += kThreads / kRowsPerCta) {
        const float v = Xs[c * kXs + q];
        const int64_t off = base + L * c;
        if (f64) reinterpret_cast<double*>(Y)[off] = (double)v; else reinterpret_cast<float*>(Y)[off] = v;
      }
    }
  }
}

constexpr size_t kSmemBytes = sizeof(float) * (TKS_MAX_BASIS * kMaxCols + TKS_MAX_BASIS * kXs);
static_assert(kMaxCols <= TKS_MAX_BASIS, "the result tile reuses the fibre tile");

}  // namespace

int ttm_rows_tiles(int64_t rows) { return (int)((rows + kRowsPerCta - 1) / kRowsPerCta); }
bool ttm_rows_fits(int b, int rmax) { return b <= TKS_MAX_BASIS && rmax <= kMaxCols; }

cudaError_t prepare_ttm_rows() {
  return cudaFuncSetAttribute(ttm_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

void launch_ttm_rows(const TtmJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream) {
  ttm_rows_kernel<<<total_tiles, kThreads, kSmemBytes, stream>>>(jobs, njobs, bases);
}

}  // namespace tks

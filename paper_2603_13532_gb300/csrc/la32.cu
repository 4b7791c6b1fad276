// Float32 small dense linear algebra of the mixed-precision path: Householder QR of the sketches
// Y_n and of the unfolded projected cores H_(n)^T, and a one-sided Jacobi SVD of the triangular
// factor.  Both are backward stable without forming Gram matrices, so the float32 rounding
// perturbs the kept subspaces by about 1e-7 relative to ||H|| instead of squaring the spectrum.
#include <cuda_runtime.h>

#include "bf16.cuh"
#include "fastdiv.cuh"
#include "kernels.h"

namespace tks {

namespace {

__device__ __forceinline__ void record_status_la(Status* st, int code) {
  if (st) atomicCAS(&st->code, 0, code);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of kN independent values, their butterflies interleaved (one shuffle latency per
// level instead of kN).
template <int kN>
__device__ __forceinline__ void warp_sum_n(float (&v)[kN]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < kN; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
}

// Step j of the register-resident Householder sweeps: apply reflector (vj, tau) to every column
// l > j (l < ncols) that this warp holds, all slots' dot products and warp reductions interleaved.
template <int kRpl, int kSlots, int kWarps>
__device__ __forceinline__ void apply_reflector(float (&a)[kSlots][kRpl], const float (&vj)[kRpl], float tau, int j,
                                                int ncols) {
  const int warp = threadIdx.x >> 5;
  if (tau == 0.f) return;
  float dot[kSlots];
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kWarps * sl;
    float d0 = 0.f, d1 = 0.f;
    if (l > j && l < ncols) {   // warp-uniform: finished and absent columns skip the products
#pragma unroll
      for (int u = 0; u + 1 < kRpl; u += 2) {
        d0 = fmaf(vj[u], a[sl][u], d0);
        d1 = fmaf(vj[u + 1], a[sl][u + 1], d1);
      }
      if (kRpl & 1) d0 = fmaf(vj[kRpl - 1], a[sl][kRpl - 1], d0);
    }
    dot[sl] = d0 + d1;
  }
  warp_sum_n(dot);
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kWarps * sl;
    if (l > j && l < ncols) {
      const float w = tau * dot[sl];
#pragma unroll
      for (int u = 0; u < kRpl; ++u) a[sl][u] = fmaf(-w, vj[u], a[sl][u]);
    }
  }
}

__device__ float block_sum_f(float v, float* red) {
  v = warp_sum_f(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

constexpr int kLoadBatch = 8;   // global loads in flight per thread when staging a block
constexpr int kTsqrMaxRows = 512;   // rows of one TSQR block (at most; 32 x rows per lane)

__device__ __forceinline__ float load_any(const char* base, int32_t type, int64_t idx) {
  if (type == T_F64) return (float)reinterpret_cast<const double*>(base)[idx];
  if (type == T_F32) return reinterpret_cast<const float*>(base)[idx];
  const uint32_t u = (uint32_t)reinterpret_cast<const uint16_t*>(base)[idx] << 16;
  return __uint_as_float(u);
}

__global__ void __launch_bounds__(512) qr_f32_kernel(const QrF32Job* __restrict__ jobs, Bases bases, Status* status) {
  __shared__ float red[32];
  __shared__ float sh_tau, sh_scale;
  __shared__ int sh_bad;
  const QrF32Job& J = jobs[blockIdx.x];
  const int64_t n = J.rows;
  const int S = (int)J.cols, b = J.b;
  const char* src = at<char>(bases, J.src);
  float* W = at<float>(bases, J.W);
  float* tau = at<float>(bases, J.tau);
  for (int64_t e = threadIdx.x; e < n * S; e += blockDim.x) {
    const int64_t j = e / n, i = e - j * n;
    const int64_t i1 = i / J.L0, i0 = i - i1 * J.L0;
    W[e] = load_any(src, J.src_type, i0 * J.s0 + i1 * J.s1 + j * J.sc);
  }
  if (threadIdx.x == 0) sh_bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < b; ++j) {
    float* wj = W + n * j;
    float part = 0.f;
    for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) part = fmaf(wj[i], wj[i], part);
    const float tail2 = block_sum_f(part, red);
    if (threadIdx.x == 0) {
      const float alpha = wj[j];
      const float nrm = sqrtf(fmaf(alpha, alpha, tail2));
      if (!isfinite(nrm)) sh_bad = 1;
      if (tail2 == 0.f || !isfinite(nrm)) {
        sh_tau = 0.f;
        sh_scale = 0.f;
      } else {
        const float beta = (alpha >= 0.f) ? -nrm : nrm;
        sh_tau = (beta - alpha) / beta;
        sh_scale = 1.f / (alpha - beta);
        wj[j] = beta;
      }
      tau[j] = sh_tau;
    }
    __syncthreads();
    const float t = sh_tau;
    if (t != 0.f) {
      const float sc = sh_scale;
      for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) wj[i] *= sc;
    }
    __syncthreads();
    if (t != 0.f) {
      for (int l = j + 1 + warp; l < S; l += nw) {
        float* wl = W + n * l;
        float dot = 0.f;
        for (int64_t i = j + 1 + lane; i < n; i += 32) dot = fmaf(wj[i], wl[i], dot);
        dot = warp_sum_f(dot) + wl[j];
        const float w = t * dot;
        if (lane == 0) wl[j] -= w;
        for (int64_t i = j + 1 + lane; i < n; i += 32) wl[i] = fmaf(-w, wj[i], wl[i]);
      }
    }
    __syncthreads();
  }
  if (J.want_r) {
    // R is cols x cols; rows at and below b = min(rows, cols) are zero (rank <= rows)
    float* R = at<float>(bases, J.R);
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
      const int c = e / S, r = e - c * S;
      R[e] = (r <= c && r < b) ? W[r + n * c] : 0.f;
    }
  }
  if (J.want_q) {
    double* Q = at<double>(bases, J.Q);
    // Q = H_0 ... H_{b-1} [I; 0] accumulated backwards in float32 inside W's first b columns
    // is not possible (W holds the reflectors), so accumulate into Q directly in float64
    for (int64_t e = threadIdx.x; e < n * b; e += blockDim.x) {
      const int64_t c = e / n, r = e - c * n;
      Q[e] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = b - 1; j >= 0; --j) {
      const float t = tau[j];
      if (t == 0.f) continue;
      const float* vj = W + n * j;
      for (int l = j + warp; l < b; l += nw) {
        double* ql = Q + n * l;
        float dot = 0.f;
        for (int64_t i = j + 1 + lane; i < n; i += 32) dot = fmaf(vj[i], (float)ql[i], dot);
        dot = warp_sum_f(dot) + (float)ql[j];
        const float w = t * dot;
        if (lane == 0) ql[j] = (double)((float)ql[j] - w);
        for (int64_t i = j + 1 + lane; i < n; i += 32) ql[i] = (double)fmaf(-w, vj[i], (float)ql[i]);
      }
      __syncthreads();
    }
    for (int l = warp; l < b; l += nw) {
      if (W[n * l + l] < 0.f) {
        double* ql = Q + n * l;
        for (int64_t i = lane; i < n; i += 32) ql[i] = -ql[i];
      }
    }
  }
  if (threadIdx.x == 0 && sh_bad) record_status_la(status, TKS_ENONFINITE);
}



// ----------------------------------------------------------------------------- QR in shared memory
// Householder QR of Y (n x S, float64 in, float32 arithmetic) held in shared memory, then the
// explicit Q formed in place from the stored reflectors (backward accumulation: for j = b-1..0
// apply H_j to the columns right of j, then replace column j by H_j e_j), columns flipped so
// that diag(R) >= 0, written as float64.
__global__ void __launch_bounds__(1024) qr_smem_f32_kernel(const QrF32Job* __restrict__ jobs, Bases bases,
                                                           Status* status) {
  extern __shared__ float sq[];
  __shared__ int sh_bad;
  const QrF32Job& J = jobs[blockIdx.x];
  const int n = (int)J.rows, S = (int)J.cols, b = J.b;
  float* W = sq;                 // n x S, ld n
  float* tau = W + (size_t)n * S;
  float* rdiag = tau + S;
  const char* src = at<char>(bases, J.src);
  const uint32_t L0 = (uint32_t)J.L0;
  for (int e0 = 0; e0 < n * S; e0 += kLoadBatch * (int)blockDim.x) {
    float v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * blockDim.x + threadIdx.x;
      v[u] = 0.f;
      if (e < n * S) {
        const int j = e / n, i = e - j * n;
        const uint32_t i1 = (uint32_t)i / L0, i0 = (uint32_t)i - i1 * L0;
        v[u] = load_any(src, J.src_type, (int64_t)i0 * J.s0 + (int64_t)i1 * J.s1 + (int64_t)j * J.sc);
      }
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * blockDim.x + threadIdx.x;
      if (e < n * S) W[e] = v[u];
    }
  }
  if (threadIdx.x == 0) sh_bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // reflectors stay unscaled (x below the diagonal, v = (1, x / (alpha - beta))); the warp that
  // updates column j + 1 also returns its new tail norm, so each column costs one barrier
  float* vscale = rdiag + S;
  __shared__ float sh_tail[2];
  if (warp == 0) {
    float t = 0.f;
    for (int i = 1 + lane; i < n; i += 32) t = fmaf(W[i], W[i], t);
    t = warp_sum_f(t);
    if (lane == 0) sh_tail[0] = t;
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    const float* wj = W + (size_t)n * j;
    const float alpha = wj[j];
    const float tail2 = sh_tail[j & 1];
    const float nrm = sqrtf(fmaf(alpha, alpha, tail2));
    const bool reflect = tail2 > 0.f && isfinite(nrm);
    const float beta = alpha >= 0.f ? -nrm : nrm;
    const float t = reflect ? (beta - alpha) / beta : 0.f;
    const float sc = reflect ? 1.f / (alpha - beta) : 0.f;
    if (threadIdx.x == 0) {
      if (!isfinite(nrm)) sh_bad = 1;
      rdiag[j] = reflect ? beta : alpha;
      tau[j] = t;
      vscale[j] = sc;
    }
    for (int l = j + 1 + warp; l < b; l += nw) {
      float* wl = W + (size_t)n * l;
      if (reflect) {
        float dot = 0.f;
        for (int i = j + 1 + lane; i < n; i += 32) dot = fmaf(wj[i], wl[i], dot);
        dot = fmaf(warp_sum_f(dot), sc, wl[j]);
        const float w = t * dot;
        if (lane == 0) wl[j] -= w;
        const float ws = w * sc;
        for (int i = j + 1 + lane; i < n; i += 32) wl[i] = fmaf(-ws, wj[i], wl[i]);
      }
      if (l == j + 1) {
        __syncwarp();   // the column's update by other lanes is visible
        float tt = 0.f;
        for (int i = j + 2 + lane; i < n; i += 32) tt = fmaf(wl[i], wl[i], tt);
        tt = warp_sum_f(tt);
        if (lane == 0) sh_tail[(j + 1) & 1] = tt;
      }
    }
    __syncthreads();
  }
  // explicit Q in place (columns 0..b-1), v_j = (1, vscale_j x_j)
  for (int j = b - 1; j >= 0; --j) {
    const float t = tau[j], sc = vscale[j];
    float* wj = W + (size_t)n * j;
    if (t != 0.f) {
      for (int l = j + 1 + warp; l < b; l += nw) {
        float* wl = W + (size_t)n * l;
        float dot = 0.f;
        for (int i = j + 1 + lane; i < n; i += 32) dot = fmaf(wj[i], wl[i], dot);
        dot = fmaf(warp_sum_f(dot), sc, wl[j]);
        const float w = t * dot;
        if (lane == 0) wl[j] -= w;
        const float ws = w * sc;
        for (int i = j + 1 + lane; i < n; i += 32) wl[i] = fmaf(-ws, wj[i], wl[i]);
      }
    }
    __syncthreads();
    const float tv = t * sc;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (i < j) wj[i] = 0.f;
      else if (i == j) wj[i] = 1.f - t;
      else wj[i] = -tv * wj[i];
    }
    __syncthreads();
  }
  double* Q = at<double>(bases, J.Q);
  for (int e = threadIdx.x; e < n * b; e += blockDim.x) {
    const int l = e / n;
    const float sgn = rdiag[l] < 0.f ? -1.f : 1.f;
    Q[e] = f32_to_f64_exact(sgn * W[e]);
  }
  if (threadIdx.x == 0 && sh_bad) record_status_la(status, TKS_ENONFINITE);
}

// Forms the reflector of column c (owned by this warp, values a[u] at rows lane + 32 u, m rows)
// below row c and publishes v (entries [0, vlen)), tau and the diagonal entry of R; returns
// false when the column norm is not finite.
template <int kRpl>
__device__ __forceinline__ bool reflector_publish(const float (&a)[kRpl], int c, int m, float* v_out, int vlen,
                                                  float* tau_out, float* rdiag) {
  const int lane = threadIdx.x & 31;
  float t2 = 0.f, alpha = 0.f;
#pragma unroll
  for (int u = 0; u < kRpl; ++u) {
    const int i = lane + 32 * u;
    if (i > c && i < m) t2 = fmaf(a[u], a[u], t2);
    if (i == c) alpha = a[u];
  }
  t2 = warp_sum_f(t2);
  alpha = __shfl_sync(0xffffffffu, alpha, c & 31);
  const float nrm = sqrtf(fmaf(alpha, alpha, t2));
  const bool reflect = t2 > 0.f && isfinite(nrm);
  const float beta = alpha >= 0.f ? -nrm : nrm;
  const float tau = reflect ? (beta - alpha) / beta : 0.f;
  const float sc = reflect ? 1.f / (alpha - beta) : 0.f;
#pragma unroll
  for (int u = 0; u < kRpl; ++u) {
    const int i = lane + 32 * u;
    if (i < vlen) v_out[i] = i < c ? 0.f : (i == c ? 1.f : (i < m ? sc * a[u] : 0.f));
  }
  if (lane == 0) {
    *tau_out = tau;
    rdiag[c] = reflect ? beta : alpha;
  }
  return isfinite(nrm);
}

// ----------------------------------------------------------------------------- QR in registers
// Householder QR of Y (n x S, n <= 32 kRpl, S <= 16 kSlots) with the explicit Q (first b columns),
// float32 arithmetic, float64 in and out.  Y is staged through shared memory and then held in
// registers as in the TSQR block kernel (column l in warp l % 16, rows lane + 32 u); reflector j
// is published into column j of the staging buffer, which afterwards holds all of them, so the
// columns of Q = H_0 .. H_{b-1} [I_b; 0] are formed without further barriers (column l needs
// H_l .. H_0 applied to e_l).  Columns are flipped so that diag(R) >= 0.
constexpr int kQrRegThreads = 512;
constexpr int kQrRegWarps = kQrRegThreads / 32;

template <int kRpl, int kSlots>
__global__ void __launch_bounds__(kQrRegThreads, 1) qr_reg_f32_kernel(const QrF32Job* __restrict__ jobs, Bases bases,
                                                                     Status* status) {
  extern __shared__ float vs[];            // n x S: Y staged, then reflector j in column j
  __shared__ float tau_s[TKS_MAX_BASIS];
  __shared__ float rdiag_s[TKS_MAX_BASIS];
  __shared__ int sh_bad;
  const QrF32Job& J = jobs[blockIdx.x];
  const int n = (int)J.rows, S = (int)J.cols, b = J.b;
  const char* src = at<char>(bases, J.src);
  const uint32_t L0 = (uint32_t)J.L0;
  const SmallDiv dn(n), dl0((int)L0);   // n <= 512, L0 <= n, e < n S <= 2^15
  if (threadIdx.x == 0) sh_bad = 0;
  for (int e0 = 0; e0 < n * S; e0 += kLoadBatch * kQrRegThreads) {
    float v[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * kQrRegThreads + threadIdx.x;
      v[u] = 0.f;
      if (e < n * S) {
        const int j = dn.quo(e), i = e - j * n;
        const uint32_t i1 = (uint32_t)dl0.quo(i), i0 = (uint32_t)i - i1 * L0;
        v[u] = load_any(src, J.src_type, (int64_t)i0 * J.s0 + (int64_t)i1 * J.s1 + (int64_t)j * J.sc);
      }
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * kQrRegThreads + threadIdx.x;
      if (e < n * S) vs[e] = v[u];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float a[kSlots][kRpl];
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kQrRegWarps * sl;
#pragma unroll
    for (int u = 0; u < kRpl; ++u) {
      const int i = lane + 32 * u;
      a[sl][u] = (l < S && i < n) ? vs[i + n * l] : 0.f;
    }
  }
  __syncthreads();   // the staging buffer now receives the reflectors
  bool bad = false;
  if (warp == 0 && b > 0) bad |= !reflector_publish(a[0], 0, n, vs, n, &tau_s[0], rdiag_s);
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    const float tau = tau_s[j];
    float vj[kRpl];
#pragma unroll
    for (int u = 0; u < kRpl; ++u) {
      const int i = lane + 32 * u;
      vj[u] = i < n ? vs[i + n * j] : 0.f;
    }
    apply_reflector<kRpl, kSlots, kQrRegWarps>(a, vj, tau, j, S);
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
      const int l = warp + kQrRegWarps * sl;
      if (l == j + 1 && l < b) bad |= !reflector_publish(a[sl], l, n, vs + n * l, n, &tau_s[l], rdiag_s);
    }
    __syncthreads();
  }
  if (bad && lane == 0) sh_bad = 1;
  // Q: column l = H_0 .. H_l e_l, reflectors read from shared memory
  double* Q = at<double>(bases, J.Q);
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kQrRegWarps * sl;
    if (l < b) {
      float q[kRpl];
#pragma unroll
      for (int u = 0; u < kRpl; ++u) q[u] = (lane + 32 * u == l) ? 1.f : 0.f;
      for (int jj = l; jj >= 0; --jj) {
        const float t = tau_s[jj];
        if (t == 0.f) continue;
        float v[kRpl];
        float dot = 0.f;
#pragma unroll
        for (int u = 0; u < kRpl; ++u) {
          const int i = lane + 32 * u;
          v[u] = i < n ? vs[i + n * jj] : 0.f;
          dot = fmaf(v[u], q[u], dot);
        }
        const float w = t * warp_sum_f(dot);
#pragma unroll
        for (int u = 0; u < kRpl; ++u) q[u] = fmaf(-w, v[u], q[u]);
      }
      const float sgn = rdiag_s[l] < 0.f ? -1.f : 1.f;
#pragma unroll
      for (int u = 0; u < kRpl; ++u) {
        const int i = lane + 32 * u;
        if (i < n) {
          const float v = sgn * q[u];
          Q[i + (int64_t)n * l] = f32_to_f64_exact(v);
          if (J.nplanes) {
            // the same planes the float64 -> bf16 split gives for this float32 value
            uint16_t h0, h1, h2;
            split3(v, h0, h1, h2);
            at<uint16_t>(bases, J.Qp[0])[i + (int64_t)n * l] = h0;
            at<uint16_t>(bases, J.Qp[1])[i + (int64_t)n * l] = h1;
            at<uint16_t>(bases, J.Qp[2])[i + (int64_t)n * l] = h2;
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && sh_bad) record_status_la(status, TKS_ENONFINITE);
}

// ----------------------------------------------------------------------------- TSQR block
// Householder QR of a rows x cols block (rows <= 256, cols <= 32 kSlots), only the triangular
// factor kept.  The block is staged through shared memory once and then lives in registers:
// column l belongs to warp l % 16 (slot l / 16), lane L holds rows L + 32 u, u < 8.  Step j
// reads the published reflector v_j = (0, .., 0, 1, x / (alpha - beta)) and tau_j from shared
// memory; every warp updates its columns l > j in registers (a_l -= tau v (v^T a_l), one warp
// reduction per column), and the warp owning column j + 1 then forms that column's reflector
// and publishes it, so each column costs one barrier and no shared-memory traffic for the
// trailing matrix.
constexpr int kTsqrThreads = 512;
constexpr int kTsqrWarps = kTsqrThreads / 32;

template <int kTsqrRowsPerLane, int kSlots>
__global__ void __launch_bounds__(kTsqrThreads, kTsqrRowsPerLane * kSlots <= 32 ? 2 : 1)
    tsqr_f32_kernel(const TsqrJob* __restrict__ jobs, Bases bases) {
  constexpr int kBlockRows = 32 * kTsqrRowsPerLane;
  extern __shared__ float smem_t[];
  __shared__ float vbuf[2][kBlockRows];
  __shared__ float sh_tau[2];
  __shared__ float rdiag[32 * kSlots];
  __shared__ int64_t rowoff[kBlockRows];
  const TsqrJob& J = jobs[blockIdx.x];
  const int m = J.rows, b = J.cols;
  const int ld = m + 1;
  float* A = smem_t;
  const char* src = at<char>(bases, J.src);
  // source offset of each row of the block (row index i = (i0, i1) with i0 fastest)
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const uint64_t i = (uint64_t)(J.row_begin + r), L0 = (uint64_t)J.L0;
    const uint64_t i1 = i / L0, i0 = i - i1 * L0;
    rowoff[r] = (int64_t)i0 * J.s0 + (int64_t)i1 * J.s1;
  }
  __syncthreads();
  // stage: columns fastest when a row is contiguous in the source, else rows; kLoadBatch loads
  // in flight per thread before the shared-memory stores
  const bool row_major = J.sc == 1;
  const int mb = m * b;   // <= 2^15 (m <= 512 when b <= 64, else m <= 256)
  const SmallDiv dq(row_major ? b : m);
  for (int e0 = 0; e0 < mb; e0 += kLoadBatch * kTsqrThreads) {
    float v[kLoadBatch];
    int dst[kLoadBatch];
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int e = e0 + u * kTsqrThreads + threadIdx.x;
      v[u] = 0.f;
      dst[u] = -1;
      if (e < mb) {
        const int q = dq.quo(e);
        const int r = row_major ? q : e - q * m, c = row_major ? e - q * b : q;
        v[u] = load_any(src, J.src_type, rowoff[r] + (int64_t)c * J.sc);
        dst[u] = r + ld * c;
      }
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u)
      if (dst[u] >= 0) A[dst[u]] = v[u];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float a[kSlots][kTsqrRowsPerLane];
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kTsqrWarps * sl;
#pragma unroll
    for (int u = 0; u < kTsqrRowsPerLane; ++u) {
      const int i = lane + 32 * u;
      a[sl][u] = (l < b && i < m) ? A[i + ld * l] : 0.f;
    }
  }
  const int kmax = m < b ? m : b;
  if (warp == 0 && kmax > 0) reflector_publish(a[0], 0, m, vbuf[0], kBlockRows, &sh_tau[0], rdiag);
  __syncthreads();
  for (int j = 0; j < kmax; ++j) {
    const float tau = sh_tau[j & 1];
    float vj[kTsqrRowsPerLane];
#pragma unroll
    for (int u = 0; u < kTsqrRowsPerLane; ++u) vj[u] = vbuf[j & 1][lane + 32 * u];
    apply_reflector<kTsqrRowsPerLane, kSlots, kTsqrWarps>(a, vj, tau, j, b);
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
      const int l = warp + kTsqrWarps * sl;
      if (l == j + 1 && l < kmax)
        reflector_publish(a[sl], l, m, vbuf[(j + 1) & 1], kBlockRows, &sh_tau[(j + 1) & 1], rdiag);
    }
    __syncthreads();
  }
  // R: row r < c of column c from the owner's registers, the diagonal from rdiag, zeros below
  float* dst = at<float>(bases, J.dst);
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int c = warp + kTsqrWarps * sl;
    if (c < b) {
#pragma unroll
      for (int u = 0; u < kTsqrRowsPerLane; ++u) {
        const int r = lane + 32 * u;
        if (r < b) {
          float v = 0.f;
          if (r < kmax && r <= c) v = (r == c) ? rdiag[r] : a[sl][u];
          dst[(J.dst_row0 + r) + J.dst_ld * c] = v;
        }
      }
    }
  }
}

// One-sided Jacobi on the columns of the b x b matrix A = R with the round-robin ordering:
// each round rotates b/2 disjoint column pairs (kSvdLanes lanes per pair) so that they become
// orthogonal; V accumulates the rotations.  At convergence A = U Sigma, R = U Sigma V^T.
constexpr int kSvdSweeps = 30;
constexpr int kSvdLanes = 8;      // lanes per column pair
constexpr int kSvdThreads = 384;  // kSvdLanes x (TKS_MAX_BASIS / 2) pairs, at most
constexpr int kSvdChunks = (TKS_MAX_BASIS + 4 * kSvdLanes - 1) / (4 * kSvdLanes);   // 4-row chunks per lane

__global__ void __launch_bounds__(kSvdThreads) svd_jacobi_f32_kernel(const SvdJob* __restrict__ jobs, Bases bases,
                                                              Status* status) {
  extern __shared__ float sm[];
  const SvdJob& J = jobs[blockIdx.x];
  const int b = J.b;
  const int m = b + (b & 1);
  const int ld = (m + 3) & ~3;   // columns start 16-byte aligned; rows in [b, ld) stay zero
  float* A = sm;
  float* V = A + m * ld;
  float* nrm = V + m * ld;
  int* order = reinterpret_cast<int*>(nrm + m);
  __shared__ int sh_rot, sh_rank;
  __shared__ float red[32];
  const float* Rg = at<float>(bases, J.R);
  for (int e = threadIdx.x; e < m * ld; e += blockDim.x) {
    const int r = e % ld, c = e / ld;
    A[e] = (r < b && c < b) ? Rg[r + c * b] : 0.f;
    V[e] = (r == c) ? 1.f : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // rotate while |a_p . a_q| > b eps_f32 ||a_p|| ||a_q|| (the usual m eps convergence test), except
  // for columns at the float32 noise floor (norm <= 8 eps max column norm): their couplings are
  // rounding noise that the relative test would chase forever, and they cannot be resolved anyway
  const float thr = (float)b * 5.96e-8f;
  __shared__ float sh_noise2;
  {
    if (threadIdx.x == 0) sh_noise2 = 0.f;
    __syncthreads();
    for (int c = warp; c < b; c += nw) {
      float s2 = 0.f;
      for (int i = lane; i < b; i += 32) s2 = fmaf(A[i + c * ld], A[i + c * ld], s2);
      s2 = warp_sum_f(s2);
      if (lane == 0) atomicMax(reinterpret_cast<int*>(&sh_noise2), __float_as_int(s2));
    }
    __syncthreads();
    if (threadIdx.x == 0) sh_noise2 *= (8.f * 5.96e-8f) * (8.f * 5.96e-8f);
    __syncthreads();
  }
  const float noise2 = sh_noise2;
  // a group of kSvdLanes lanes rotates one pair; pair k of a round is (round + k, round - k) mod
  // (m - 1), pair 0 is (round, m - 1)
  const int sub = lane % kSvdLanes;
  const int k = (threadIdx.x / kSvdLanes);
  const int pairs = m / 2;
  int sweep = 0;
  for (; sweep < kSvdSweeps; ++sweep) {
    if (threadIdx.x == 0) sh_rot = 0;
    __syncthreads();
    int any = 0;
    for (int round = 0; round < m - 1; ++round) {
      int p = 0, q = 0;
      if (k == 0) {
        p = round;
        q = m - 1;
      } else {
        p = round + k;
        if (p >= m - 1) p -= m - 1;
        q = round - k;
        if (q < 0) q += m - 1;
      }
      if (p > q) { const int t = p; p = q; q = t; }
      const bool valid = k < pairs && q < b;
      if (!valid) p = q = 0;
      float* ap = A + p * ld;
      float* aq = A + q * ld;
      // lane `sub` of the group holds the 4-row chunks sub, sub + 8, ... of both columns
      float4 x[kSvdChunks], y[kSvdChunks];
      float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
      for (int u = 0; u < kSvdChunks; ++u) {
        const int i = 4 * (sub + kSvdLanes * u);
        const bool in = valid && i < b;
        x[u] = in ? *reinterpret_cast<const float4*>(ap + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        y[u] = in ? *reinterpret_cast<const float4*>(aq + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kSvdChunks; ++u) {
        al = fmaf(x[u].x, x[u].x, fmaf(x[u].y, x[u].y, fmaf(x[u].z, x[u].z, fmaf(x[u].w, x[u].w, al))));
        be = fmaf(y[u].x, y[u].x, fmaf(y[u].y, y[u].y, fmaf(y[u].z, y[u].z, fmaf(y[u].w, y[u].w, be))));
        ga = fmaf(x[u].x, y[u].x, fmaf(x[u].y, y[u].y, fmaf(x[u].z, y[u].z, fmaf(x[u].w, y[u].w, ga))));
      }
      // every lane takes part in the group reductions
#pragma unroll
      for (int o = kSvdLanes / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o, kSvdLanes);
        be += __shfl_xor_sync(0xffffffffu, be, o, kSvdLanes);
        ga += __shfl_xor_sync(0xffffffffu, ga, o, kSvdLanes);
      }
      if (valid && fabsf(ga) > thr * sqrtf(al * be) && ga != 0.f && fminf(al, be) > noise2) {
        // the angle only steers convergence, so t is formed with fast division; the rotation's
        // orthogonality rests on c^2 + s^2 = 1, so c = 1 / sqrt(1 + t^2) gets a Newton step
        const float zeta = __fdividef(be - al, 2.f * ga);
        const float az = fabsf(zeta);
        const float tm = az > 1e18f ? __fdividef(0.5f, az) : __fdividef(1.f, az + sqrtf(fmaf(az, az, 1.f)));
        const float t = copysignf(tm, zeta);
        const float w = fmaf(t, t, 1.f);
        float c = rsqrtf(w);
        c = c * fmaf(-0.5f * w * c, c, 1.5f);
        const float s = c * t;
        float* vp = V + p * ld;
        float* vq = V + q * ld;
#pragma unroll
        for (int u = 0; u < kSvdChunks; ++u) {
          const int i = 4 * (sub + kSvdLanes * u);
          if (i < b) {
            const float4 a = x[u], bb = y[u];
            *reinterpret_cast<float4*>(ap + i) =
                make_float4(c * a.x - s * bb.x, c * a.y - s * bb.y, c * a.z - s * bb.z, c * a.w - s * bb.w);
            *reinterpret_cast<float4*>(aq + i) =
                make_float4(s * a.x + c * bb.x, s * a.y + c * bb.y, s * a.z + c * bb.z, s * a.w + c * bb.w);
            const float4 vx = *reinterpret_cast<const float4*>(vp + i);
            const float4 vy = *reinterpret_cast<const float4*>(vq + i);
            *reinterpret_cast<float4*>(vp + i) =
                make_float4(c * vx.x - s * vy.x, c * vx.y - s * vy.y, c * vx.z - s * vy.z, c * vx.w - s * vy.w);
            *reinterpret_cast<float4*>(vq + i) =
                make_float4(s * vx.x + c * vy.x, s * vx.y + c * vy.y, s * vx.z + c * vy.z, s * vx.w + c * vy.w);
          }
        }
        any = 1;
      }
      __syncthreads();
    }
    if (any) sh_rot = 1;
    __syncthreads();
    const int rot = sh_rot;
    __syncthreads();
    if (!rot) break;
  }
  // singular values = column norms; sort descending
  for (int c = warp; c < b; c += nw) {
    float s = 0.f;
    for (int i = lane; i < b; i += 32) s = fmaf(A[i + c * ld], A[i + c * ld], s);
    s = warp_sum_f(s);
    if (lane == 0) nrm[c] = s;
  }
  __syncthreads();
  float tot = 0.f;
  {
    float part = 0.f;
    for (int i = threadIdx.x; i < b; i += blockDim.x) part += nrm[i];
    tot = block_sum_f(part, red);
  }
  // columns by decreasing norm: thread i places column i at its rank (ties by index; a NaN norm
  // counts as -1, so the ranks always form a permutation); a serial selection sort here cost
  // b^2 / 2 dependent shared-memory reads in one thread
  if ((int)threadIdx.x < b) {
    const int i = threadIdx.x;
    const float ni = nrm[i] == nrm[i] ? nrm[i] : -1.f;
    int rk = 0;
    for (int j = 0; j < b; ++j) {
      const float nj = nrm[j] == nrm[j] ? nrm[j] : -1.f;
      rk += (nj > ni || (nj == ni && j < i)) ? 1 : 0;
    }
    order[rk] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float* sv = at<float>(bases, J.sv);
    for (int i = 0; i < b; ++i) sv[i] = sqrtf(nrm[order[i]]);
    double* theta = at<double>(bases, J.theta);
    if (J.first_mode) *theta = J.tol * J.tol * (double)tot / J.order;
    int r = J.rmax;
    if (J.tol > 0.0) {
      const double th = *theta;
      double tail = 0.0;
      r = b;
      for (int i = b - 1; i >= 1; --i) {
        tail += nrm[order[i]];
        if (tail <= th) r = i; else break;
      }
      if (r > J.rmax) r = J.rmax;
    }
    sh_rank = r;
    if (J.err.base != B_NONE) {
      // the energy this mode's truncation discards; with the first mode's total, the ST-HOSVD's
      // relative error (the discarded parts of successive modes are orthogonal)
      double* er = at<double>(bases, J.err);
      double dis = 0.0;
      for (int i = r; i < b; ++i) dis += (double)nrm[order[i]];
      if (J.first_mode) er[0] = (double)tot;
      er[1 + J.mode] = dis;
    }
    *at<int32_t>(bases, J.rank) = r;
    if (!isfinite(tot)) record_status_la(status, TKS_ENONFINITE);
    if (sweep >= kSvdSweeps) record_status_la(status, TKS_ENOCONV);
  }
  __syncthreads();
  const int r = sh_rank;
  // The kept right singular vectors, sign-fixed (largest entry positive), into the A buffer
  // (column t at A + t ld).  V comes out of some b x sweeps plane rotations per column, each
  // orthogonal to float32 rounding, so its columns drift from orthonormality by about
  // b sweeps eps (5e-5 for b = 64); one Newton-Schulz step P <- P (3 I - P^T P) / 2, which keeps
  // span(P) and squares the deviation, restores it to rounding level.
  for (int t = warp; t < r; t += nw) {
    const int src = order[t];
    float best = 0.f;
    for (int i = lane; i < b; i += 32) {
      const float v = V[i + src * ld];
      if (fabsf(v) > fabsf(best)) best = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float other = __shfl_xor_sync(0xffffffffu, best, o);
      if (fabsf(other) > fabsf(best) || (fabsf(other) == fabsf(best) && other > best)) best = other;
    }
    const float sgn = (best < 0.f) ? -1.f : 1.f;
    for (int i = lane; i < b; i += 32) A[i + t * ld] = sgn * V[i + src * ld];
  }
  __syncthreads();
  // G = P^T P into the V buffer (G[t1 + t2 ld])
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int t1 = e % r, t2 = e / r;
    const float* p1 = A + t1 * ld;
    const float* p2 = A + t2 * ld;
    float acc = 0.f;
    for (int i = 0; i < b; ++i) acc = fmaf(p1[i], p2[i], acc);
    V[t1 + t2 * ld] = acc;
  }
  __syncthreads();
  float* P = at<float>(bases, J.P);
  for (int e = threadIdx.x; e < b * J.rmax; e += blockDim.x) {
    const int i = e % b, t = e / b;
    float v = 0.f;
    if (t < r) {
      float acc = 0.f;
      for (int t2 = 0; t2 < r; ++t2) acc = fmaf(A[i + t2 * ld], V[t2 + t * ld], acc);
      v = fmaf(1.5f, A[i + t * ld], -0.5f * acc);
    }
    P[i + t * b] = v;
  }
}

size_t svd_smem(int bmax) {
  const int m = bmax + (bmax & 1), ld = (m + 3) & ~3;
  return (size_t)2 * m * ld * sizeof(float) + (size_t)m * sizeof(float) + (size_t)m * sizeof(int);
}

}  // namespace

size_t tsqr_smem(int rows, int cols) { return (size_t)(rows + 1) * cols * sizeof(float); }

cudaError_t prepare_qr_reg_f32() {
  cudaError_t e = cudaFuncSetAttribute(qr_reg_f32_kernel<4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(qr_reg_f32_kernel<8, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(qr_reg_f32_kernel<16, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t prepare_tsqr_f32() {
  cudaError_t e = cudaFuncSetAttribute(qr_smem_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 222 * 1024);
  if (e != cudaSuccess) return e;
  const void* kernels[] = {
      reinterpret_cast<const void*>(tsqr_f32_kernel<8, 2>), reinterpret_cast<const void*>(tsqr_f32_kernel<8, 3>),
      reinterpret_cast<const void*>(tsqr_f32_kernel<8, 4>), reinterpret_cast<const void*>(tsqr_f32_kernel<8, 6>),
      reinterpret_cast<const void*>(tsqr_f32_kernel<16, 2>), reinterpret_cast<const void*>(tsqr_f32_kernel<16, 3>),
      reinterpret_cast<const void*>(tsqr_f32_kernel<16, 4>)};
  for (const void* k : kernels) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t qr_smem_bytes(int64_t n, int S) { return (size_t)(n * S + 3 * S) * sizeof(float); }

void launch_qr_smem_f32(const QrF32Job* jobs, int njobs, size_t smem, const Bases& bases, Status* status,
                        cudaStream_t stream) {
  qr_smem_f32_kernel<<<njobs, 1024, smem, stream>>>(jobs, bases, status);
}

void launch_tsqr_f32(const TsqrJob* jobs, int njobs, int max_rows, int max_cols, const Bases& bases,
                     cudaStream_t stream) {
  // rows per lane and columns per warp: the smallest instantiation that covers the block
  const size_t smem = tsqr_smem(max_rows, max_cols);
  const int slots = max_cols <= 2 * kTsqrWarps ? 2 : max_cols <= 3 * kTsqrWarps ? 3 : max_cols <= 4 * kTsqrWarps ? 4 : 6;
  if (max_rows <= 256) {
    if (slots == 2) tsqr_f32_kernel<8, 2><<<njobs, kTsqrThreads, smem, stream>>>(jobs, bases);
    else if (slots == 3) tsqr_f32_kernel<8, 3><<<njobs, kTsqrThreads, smem, stream>>>(jobs, bases);
    else if (slots == 4) tsqr_f32_kernel<8, 4><<<njobs, kTsqrThreads, smem, stream>>>(jobs, bases);
    else tsqr_f32_kernel<8, 6><<<njobs, kTsqrThreads, smem, stream>>>(jobs, bases);
  } else {
    if (slots == 2) tsqr_f32_kernel<16, 2><<<njobs, kTsqrThreads, smem, stream>>>(jobs, bases);
    else if (slots == 3) tsqr_f32_kernel<16, 3><<<njobs, kTsqrThreads, smem, stream>>>(jobs, bases);
    else tsqr_f32_kernel<16, 4><<<njobs, kTsqrThreads, smem, stream>>>(jobs, bases);
  }
}

int tsqr_block_rows(int max_cols) { return max_cols <= 4 * kTsqrWarps ? 512 : 256; }

size_t qr_reg_smem_bytes(int64_t n, int S) { return (size_t)(n * S) * sizeof(float); }

bool qr_reg_fits(int64_t n, int S) { return n <= 512 && S <= 4 * kQrRegWarps && qr_reg_smem_bytes(n, S) <= 200 * 1024; }

void launch_qr_reg_f32(const QrF32Job* jobs, int njobs, int max_rows, size_t smem, const Bases& bases,
                       Status* status, cudaStream_t stream) {
  if (max_rows <= 128)
    qr_reg_f32_kernel<4, 4><<<njobs, kQrRegThreads, smem, stream>>>(jobs, bases, status);
  else if (max_rows <= 256)
    qr_reg_f32_kernel<8, 4><<<njobs, kQrRegThreads, smem, stream>>>(jobs, bases, status);
  else
    qr_reg_f32_kernel<16, 4><<<njobs, kQrRegThreads, smem, stream>>>(jobs, bases, status);
}

void launch_qr_f32(const QrF32Job* jobs, int njobs, const Bases& bases, Status* status, cudaStream_t stream) {
  qr_f32_kernel<<<njobs, 512, 0, stream>>>(jobs, bases, status);
}

cudaError_t prepare_svd_f32(int bmax) {
  return cudaFuncSetAttribute(svd_jacobi_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)svd_smem(bmax));
}

void launch_svd_f32(const SvdJob* jobs, int njobs, int bmax, const Bases& bases, Status* status,
                    cudaStream_t stream) {
  // kSvdLanes lanes per column pair of a round, whole warps: ceil(bmax / 2) <= 48 pairs
  const int pairs = (bmax + 1) / 2;
  const int threads = ((pairs * kSvdLanes + 31) / 32) * 32;
  svd_jacobi_f32_kernel<<<njobs, threads, svd_smem(bmax), stream>>>(jobs, bases, status);
}

}  // namespace tks

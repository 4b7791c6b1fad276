// Float32 small dense linear algebra of the mixed-precision path: Householder QR of the sketches
// Y_n and of the unfolded projected cores H_(n)^T, and a one-sided Jacobi SVD of the triangular
// factor.  Both are backward stable without forming Gram matrices, so the float32 rounding
// perturbs the kept subspaces by about 1e-7 relative to ||H|| instead of squaring the spectrum.
#include <cuda_runtime.h>

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
  __shared__ float red[32];
  __shared__ float sh_tau, sh_scale;
  __shared__ int sh_bad;
  const QrF32Job& J = jobs[blockIdx.x];
  const int n = (int)J.rows, S = (int)J.cols, b = J.b;
  float* W = sq;                 // n x S, ld n
  float* tau = W + (size_t)n * S;
  float* rdiag = tau + S;
  const char* src = at<char>(bases, J.src);
  for (int e = threadIdx.x; e < n * S; e += blockDim.x) {
    const int j = e / n, i = e - j * n;
    const int64_t i1 = i / J.L0, i0 = i - i1 * J.L0;
    W[e] = load_any(src, J.src_type, i0 * J.s0 + i1 * J.s1 + j * J.sc);
  }
  if (threadIdx.x == 0) sh_bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < b; ++j) {
    float* wj = W + (size_t)n * j;
    float part = 0.f;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) part = fmaf(wj[i], wj[i], part);
    const float tail2 = block_sum_f(part, red);
    if (threadIdx.x == 0) {
      const float alpha = wj[j];
      const float nrm = sqrtf(fmaf(alpha, alpha, tail2));
      if (!isfinite(nrm)) sh_bad = 1;
      if (tail2 == 0.f || !isfinite(nrm)) {
        sh_tau = 0.f;
        sh_scale = 0.f;
        rdiag[j] = alpha;
      } else {
        const float beta = (alpha >= 0.f) ? -nrm : nrm;
        sh_tau = (beta - alpha) / beta;
        sh_scale = 1.f / (alpha - beta);
        rdiag[j] = beta;
      }
      tau[j] = sh_tau;
    }
    __syncthreads();
    const float t = sh_tau;
    if (t != 0.f) {
      const float sc = sh_scale;
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) wj[i] *= sc;
      __syncthreads();
      for (int l = j + 1 + warp; l < b; l += nw) {
        float* wl = W + (size_t)n * l;
        float dot = 0.f;
        for (int i = j + 1 + lane; i < n; i += 32) dot = fmaf(wj[i], wl[i], dot);
        dot = warp_sum_f(dot) + wl[j];
        const float w = t * dot;
        if (lane == 0) wl[j] -= w;
        for (int i = j + 1 + lane; i < n; i += 32) wl[i] = fmaf(-w, wj[i], wl[i]);
      }
    }
    __syncthreads();
  }
  // explicit Q in place (columns 0..b-1)
  for (int j = b - 1; j >= 0; --j) {
    const float t = tau[j];
    float* wj = W + (size_t)n * j;
    if (t != 0.f) {
      for (int l = j + 1 + warp; l < b; l += nw) {
        float* wl = W + (size_t)n * l;
        float dot = 0.f;
        for (int i = j + 1 + lane; i < n; i += 32) dot = fmaf(wj[i], wl[i], dot);
        dot = warp_sum_f(dot) + wl[j];
        const float w = t * dot;
        if (lane == 0) wl[j] -= w;
        for (int i = j + 1 + lane; i < n; i += 32) wl[i] = fmaf(-w, wj[i], wl[i]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (i < j) wj[i] = 0.f;
      else if (i == j) wj[i] = 1.f - t;
      else wj[i] = -t * wj[i];
    }
    __syncthreads();
  }
  double* Q = at<double>(bases, J.Q);
  for (int e = threadIdx.x; e < n * b; e += blockDim.x) {
    const int l = e / n;
    const float sgn = rdiag[l] < 0.f ? -1.f : 1.f;
    Q[e] = (double)(sgn * W[e]);
  }
  if (threadIdx.x == 0 && sh_bad) record_status_la(status, TKS_ENONFINITE);
}

// ----------------------------------------------------------------------------- TSQR block
// Householder QR of a rows x cols block held in shared memory (column-major, ld = rows + 1),
// one thread block; only the triangular factor is kept.
__global__ void __launch_bounds__(512) tsqr_f32_kernel(const TsqrJob* __restrict__ jobs, Bases bases) {
  extern __shared__ float smem_t[];
  __shared__ float red[32];
  __shared__ float sh_tau, sh_scale;
  const TsqrJob& J = jobs[blockIdx.x];
  const int m = J.rows, b = J.cols;
  const int ld = m + 1;
  float* A = smem_t;
  const char* src = at<char>(bases, J.src);
  for (int e = threadIdx.x; e < m * b; e += blockDim.x) {
    const int c = e / m, r = e - c * m;
    const int64_t i = J.row_begin + r;
    const int64_t i1 = i / J.L0, i0 = i - i1 * J.L0;
    A[r + ld * c] = load_any(src, J.src_type, i0 * J.s0 + i1 * J.s1 + c * J.sc);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int kmax = m < b ? m : b;
  for (int j = 0; j < kmax; ++j) {
    float* aj = A + ld * j;
    float part = 0.f;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) part = fmaf(aj[i], aj[i], part);
    const float tail2 = block_sum_f(part, red);
    if (threadIdx.x == 0) {
      const float alpha = aj[j];
      const float nrm = sqrtf(fmaf(alpha, alpha, tail2));
      if (tail2 == 0.f || !isfinite(nrm)) {
        sh_tau = 0.f;
        sh_scale = 0.f;
      } else {
        const float beta = (alpha >= 0.f) ? -nrm : nrm;
        sh_tau = (beta - alpha) / beta;
        sh_scale = 1.f / (alpha - beta);
        aj[j] = beta;
      }
    }
    __syncthreads();
    const float t = sh_tau;
    if (t != 0.f) {
      const float sc = sh_scale;
      for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) aj[i] *= sc;
      __syncthreads();
      for (int l = j + 1 + warp; l < b; l += nw) {
        float* al = A + ld * l;
        float dot = 0.f;
        for (int i = j + 1 + lane; i < m; i += 32) dot = fmaf(aj[i], al[i], dot);
        dot = warp_sum_f(dot) + al[j];
        const float w = t * dot;
        if (lane == 0) al[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) al[i] = fmaf(-w, aj[i], al[i]);
      }
    }
    __syncthreads();
  }
  float* dst = at<float>(bases, J.dst);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int c = e / b, r = e - c * b;
    dst[(J.dst_row0 + r) + J.dst_ld * c] = (r <= c && r < kmax) ? A[r + ld * c] : 0.f;
  }
}

// One-sided Jacobi on the columns of the b x b matrix A = R with the round-robin ordering:
// each round rotates b/2 disjoint column pairs (one warp per pair) so that they become
// orthogonal; V accumulates the rotations.  At convergence A = U Sigma, R = U Sigma V^T.
constexpr int kSvdSweeps = 30;

__global__ void __launch_bounds__(1024) svd_jacobi_f32_kernel(const SvdJob* __restrict__ jobs, Bases bases,
                                                              Status* status) {
  extern __shared__ float sm[];
  const SvdJob& J = jobs[blockIdx.x];
  const int b = J.b;
  const int m = b + (b & 1);
  const int ld = m + 1;
  float* A = sm;
  float* V = A + m * ld;
  float* nrm = V + m * ld;
  int* order = reinterpret_cast<int*>(nrm + m);
  __shared__ int sh_rot, sh_rank;
  __shared__ float red[32];
  const float* Rg = at<float>(bases, J.R);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;
    A[r + c * ld] = (r < b && c < b) ? Rg[r + c * b] : 0.f;
    V[r + c * ld] = (r == c) ? 1.f : 0.f;
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
  int sweep = 0;
  for (; sweep < kSvdSweeps; ++sweep) {
    if (threadIdx.x == 0) sh_rot = 0;
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      for (int k = warp; k < m / 2; k += nw) {
        int p, q;
        if (k == 0) { p = round; q = m - 1; }
        else { p = (round + k) % (m - 1); q = (round - k + (m - 1)) % (m - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= b) continue;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int i = lane; i < b; i += 32) {
          const float x = A[i + p * ld], y = A[i + q * ld];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
        al = warp_sum_f(al);
        be = warp_sum_f(be);
        ga = warp_sum_f(ga);
        if (fabsf(ga) > thr * sqrtf(al * be) && ga != 0.f && fminf(al, be) > noise2) {
          const float zeta = (be - al) / (2.f * ga);
          const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = 1.f / sqrtf(1.f + t * t), s = c * t;
          for (int i = lane; i < b; i += 32) {
            const float x = A[i + p * ld], y = A[i + q * ld];
            A[i + p * ld] = c * x - s * y;
            A[i + q * ld] = s * x + c * y;
            const float vx = V[i + p * ld], vy = V[i + q * ld];
            V[i + p * ld] = c * vx - s * vy;
            V[i + q * ld] = s * vx + c * vy;
          }
          if (lane == 0) sh_rot = 1;
        }
      }
      __syncthreads();
    }
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
  if (threadIdx.x == 0) {
    for (int i = 0; i < b; ++i) order[i] = i;
    for (int i = 0; i < b; ++i) {
      int best = i;
      for (int j = i + 1; j < b; ++j)
        if (nrm[order[j]] > nrm[order[best]]) best = j;
      const int t = order[i]; order[i] = order[best]; order[best] = t;
    }
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
    *at<int32_t>(bases, J.rank) = r;
    if (!isfinite(tot)) record_status_la(status, TKS_ENONFINITE);
    if (sweep >= kSvdSweeps) record_status_la(status, TKS_ENOCONV);
  }
  __syncthreads();
  const int r = sh_rank;
  float* P = at<float>(bases, J.P);
  for (int t = warp; t < J.rmax; t += nw) {
    if (t >= r) {
      for (int i = lane; i < b; i += 32) P[i + t * b] = 0.f;
      continue;
    }
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
    for (int i = lane; i < b; i += 32) P[i + t * b] = sgn * V[i + src * ld];
  }
}

size_t svd_smem(int bmax) {
  const int m = bmax + (bmax & 1);
  return (size_t)2 * m * (m + 1) * sizeof(float) + (size_t)m * sizeof(float) + (size_t)m * sizeof(int);
}

}  // namespace

size_t tsqr_smem(int rows, int cols) { return (size_t)(rows + 1) * cols * sizeof(float); }

cudaError_t prepare_tsqr_f32() {
  cudaError_t e = cudaFuncSetAttribute(qr_smem_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 222 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tsqr_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 222 * 1024);
}

size_t qr_smem_bytes(int64_t n, int S) { return (size_t)(n * S + 2 * S) * sizeof(float); }

void launch_qr_smem_f32(const QrF32Job* jobs, int njobs, size_t smem, const Bases& bases, Status* status,
                        cudaStream_t stream) {
  qr_smem_f32_kernel<<<njobs, 1024, smem, stream>>>(jobs, bases, status);
}

void launch_tsqr_f32(const TsqrJob* jobs, int njobs, int max_rows, int max_cols, const Bases& bases,
                     cudaStream_t stream) {
  tsqr_f32_kernel<<<njobs, 512, tsqr_smem(max_rows, max_cols), stream>>>(jobs, bases);
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
  // one warp per column pair of a round: b / 2 <= 48 pairs, 32 warps
  svd_jacobi_f32_kernel<<<njobs, 1024, svd_smem(bmax), stream>>>(jobs, bases, status);
}

}  // namespace tks

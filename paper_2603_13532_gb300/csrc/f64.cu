// Float64 stage kernels: the plain FP64 GPU path of the method and the Householder QR of the
// sketches that the TKS_MIXED path shares (the ST-HOSVD's TSQR and SVD are in la64.cu).
//
// GB300 runs float64 at about 1/64 of the float32 CUDA-core rate (about two FP64 FMAs per
// SM per clock), so these kernels are bound by FP64 issue, not by memory: tiles are sized
// for reuse in shared memory and every SM gets work through grouped launches over all
// problems of a plan.
#include <cuda_runtime.h>

#include "kernels.h"
#include "rng.cuh"

namespace tks {

namespace {

__device__ __forceinline__ void record_status(Status* st, int code) {
  if (st) atomicCAS(&st->code, 0, code);
}

template <typename Job>
__device__ __forceinline__ int find_job(const Job* jobs, int njobs, int64_t key) {
  // last job whose begin <= key (jobs sorted by begin)
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].begin <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ----------------------------------------------------------------------------- Omega
__global__ void omega_kernel(const OmegaJob* __restrict__ jobs, int njobs, int64_t total_blocks,
                             Bases bases, uint64_t seed) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total_blocks;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int j = find_job(jobs, njobs, g);
    const OmegaJob& J = jobs[j];
    const int64_t blk = g - J.begin;
    double* out = at<double>(bases, J.out);
    if (J.bf16) {
      // low-precision sketch: float32 draws rounded to bfloat16
      float z[4];
      rng::gaussian4_f32(seed, (uint64_t)J.problem, (uint64_t)J.mode, 0ull, (uint64_t)blk, z);
      uint16_t* plane = J.has_plane ? at<uint16_t>(bases, J.plane) : nullptr;
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int64_t e = 4 * blk + l;
        if (e < J.count) {
          const uint16_t h = rng::f32_to_bf16_bits(z[l]);
          out[e] = rng::bf16_bits_to_double(h);
          if (plane) plane[e] = h;
        }
      }
    } else {
      double z[4];
      rng::gaussian4(seed, (uint64_t)J.problem, (uint64_t)J.mode, 0ull, (uint64_t)blk, z);
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int64_t e = 4 * blk + l;
        if (e < J.count) out[e] = z[l];
      }
    }
  }
}

// ----------------------------------------------------------------------------- GEMM
constexpr int GT = 64;   // tile edge
constexpr int GK = 16;   // k step

__device__ __forceinline__ int find_tile_job(const GemmJob* jobs, int njobs, int tile) {
  const int lo = tile_job(jobs, njobs, tile);
  return lo;
}

__global__ void __launch_bounds__(256) gemm_f64_kernel(const GemmJob* __restrict__ jobs, int njobs,
                                                       Bases bases) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const GemmJob& J = jobs[find_tile_job(jobs, njobs, blockIdx.x)];
  int local = blockIdx.x - J.tile_begin;
  const int tn = local % J.tiles_n;
  local /= J.tiles_n;
  const int tm = local % J.tiles_m;
  local /= J.tiles_m;
  const int ks = local % J.ksplit;
  const int bt = local / J.ksplit;
  const int kbeg = ks * J.kchunk;
  const int kend = min(J.K, kbeg + J.kchunk);
  const double* A = at<double>(bases, J.A) + bt * J.a_b;
  const double* B = at<double>(bases, J.B) + bt * J.b_b;
  const int m0 = tm * GT, n0 = tn * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool a_mfast = (J.a_m == 1);   // choose the coalesced load order
  const bool b_kfast = (J.b_k0 == 1);
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      int i, kk;
      if (a_mfast) { i = e % GT; kk = e / GT; } else { kk = e % GK; i = e / GK; }
      const int gi = m0 + i, gk = k0 + kk;
      double v = 0.0;
      if (gi < J.M && gk < kend) {
        const int kq = gk / J.K1, kr = gk - kq * J.K1;
        v = A[gi * J.a_m + kr * J.a_k0 + kq * J.a_k1];
      }
      As[kk][i] = v;
      int jj;
      if (b_kfast) { kk = e % GK; jj = e / GK; } else { jj = e % GT; kk = e / GT; }
      const int gj = n0 + jj, gk2 = k0 + kk;
      double w = 0.0;
      if (gj < J.N && gk2 < kend) {
        const int kq = gk2 / J.K1, kr = gk2 - kq * J.K1;
        w = B[gj * J.b_n + kr * J.b_k0 + kq * J.b_k1];
      }
      Bs[kk][jj] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  if (J.ksplit == 1) {
    double* C = at<double>(bases, J.C) + bt * J.c_b;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
        if (gi < J.M && gj < J.N) {
          double* c = C + gi * J.c_m + gj * J.c_n;
          const double v = J.alpha * acc[i][j];
          *c = (J.beta != 0.0) ? fma(J.beta, *c, v) : v;
        }
      }
  } else {
    double* P = at<double>(bases, J.P);
    const int64_t mn = (int64_t)J.M * J.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = m0 + ty + 16 * i, gj = n0 + tx + 16 * j;
        if (gi < J.M && gj < J.N) P[((int64_t)ks * J.batch + bt) * mn + (int64_t)gj * J.M + gi] = acc[i][j];
      }
  }
}

__device__ __forceinline__ int find_red_job(const GemmJob* jobs, int njobs, int64_t key) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].red_begin <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void splitk_reduce_f64_kernel(const GemmJob* __restrict__ jobs, int njobs, int64_t total,
                                         Bases bases) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const GemmJob& J = jobs[find_red_job(jobs, njobs, g)];
    int64_t e = g - J.red_begin;
    const int64_t mn = (int64_t)J.M * J.N;
    const int bt = (int)(e / mn);
    e -= bt * mn;
    const int gj = (int)(e / J.M), gi = (int)(e - (int64_t)gj * J.M);
    const double* P = at<double>(bases, J.P);
    double s = 0.0;
    for (int ks = 0; ks < J.ksplit; ++ks) s += P[((int64_t)ks * J.batch + bt) * mn + e];
    double* c = at<double>(bases, J.C) + bt * J.c_b + gi * J.c_m + gj * J.c_n;
    const double v = J.alpha * s;
    *c = (J.beta != 0.0) ? fma(J.beta, *c, v) : v;
  }
}

// ----------------------------------------------------------------------------- core sketch
// V_kn(a, c) = alpha_k sum_{i_j, j != n} G_k[i with i_n = a] prod_{j != n} M_j[roff_j + i_j, col_j]
// with col_j = c (Khatri-Rao, Eq. krp_sketch_result) or the j-th digit of c in the mixed radix
// of (s_j)_{j != n}, first remaining mode fastest (Kronecker, Eq. kron_sketch_result).
__global__ void core_sketch_f64_kernel(const CoreSketchJob* __restrict__ jobs, int njobs, int64_t total,
                                       Bases bases) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const CoreSketchJob& J = jobs[find_job(jobs, njobs, g)];
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
    const double* G = at<double>(bases, J.core);
    const double* Mcol[MAXD];
    for (int t = 0; t < no; ++t) {
      const int j = others[t];
      Mcol[t] = at<double>(bases, J.M[j]) + J.roff[j] + (int64_t)J.R[j] * col[j];
    }
    const int f = others[0];
    const int rf = J.r[f], sf = st[f];
    int idx[MAXD];
    for (int t = 0; t < no; ++t) idx[t] = 0;
    int64_t goff = (int64_t)a * st[n];
    double acc = 0.0;
    while (true) {
      double prod = 1.0;
      for (int t = 1; t < no; ++t) prod *= Mcol[t][idx[t]];
      double inner = 0.0;
      const double* mf = Mcol[0];
      for (int i = 0; i < rf; ++i) inner = fma(G[goff + (int64_t)i * sf], mf[i], inner);
      acc = fma(prod, inner, acc);
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
    double* V = at<double>(bases, J.V);
    V[(J.roff[n] + a) + (int64_t)J.Rn * c] = J.alpha * acc;
  }
}

// ----------------------------------------------------------------------------- Householder QR
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];   // fixed order: deterministic
  return s;
}

// W = Y; Householder reflectors H_j = I - tau_j v_j v_j^T (v_j[j] = 1) reduce W to R;
// Q = H_0 ... H_{b-1} [I; 0]; columns of Q flipped where R_jj < 0 so that diag(R) >= 0.
__global__ void __launch_bounds__(256) qr_f64_kernel(const QrJob* __restrict__ jobs, Bases bases,
                                                     Status* status) {
  __shared__ double red[32];
  __shared__ double sh_tau, sh_scale;
  __shared__ int sh_bad;
  const QrJob& J = jobs[blockIdx.x];
  if (J.gate.base != B_NONE && *at<const int32_t>(bases, J.gate) == 0) return;
  const int n = J.n, S = J.S, b = J.b;
  const double* Y = at<double>(bases, J.Y);
  double* W = at<double>(bases, J.W);
  double* Q = at<double>(bases, J.Q);
  double* tau = at<double>(bases, J.tau);
  const int64_t ns = (int64_t)n * S;
  for (int64_t e = threadIdx.x; e < ns; e += blockDim.x) W[e] = Y[e];
  if (threadIdx.x == 0) sh_bad = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < b; ++j) {
    double* wj = W + (int64_t)n * j;
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) part = fma(wj[i], wj[i], part);
    const double tail2 = block_sum(part, red);
    if (threadIdx.x == 0) {
      const double alpha = wj[j];
      const double nrm = sqrt(fma(alpha, alpha, tail2));
      if (!isfinite(nrm)) sh_bad = 1;
      if (tail2 == 0.0 || !isfinite(nrm)) {
        sh_tau = 0.0;          // H_j = I, R_jj = alpha
        sh_scale = 0.0;
      } else {
        const double beta = (alpha >= 0.0) ? -nrm : nrm;
        sh_tau = (beta - alpha) / beta;
        sh_scale = 1.0 / (alpha - beta);
        wj[j] = beta;
      }
      tau[j] = sh_tau;
    }
    __syncthreads();
    const double t = sh_tau;
    if (t != 0.0) {
      const double sc = sh_scale;
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) wj[i] *= sc;
    }
    __syncthreads();
    if (t != 0.0) {
      for (int l = j + 1 + warp; l < S; l += nw) {
        double* wl = W + (int64_t)n * l;
        double dot = 0.0;
        for (int i = j + 1 + lane; i < n; i += 32) dot = fma(wj[i], wl[i], dot);
        dot = warp_sum(dot) + wl[j];
        const double w = t * dot;
        if (lane == 0) wl[j] -= w;
        for (int i = j + 1 + lane; i < n; i += 32) wl[i] = fma(-w, wj[i], wl[i]);
      }
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{b-1} [I_b; 0], accumulated backwards
  for (int64_t e = threadIdx.x; e < (int64_t)n * b; e += blockDim.x) {
    const int col = (int)(e / n), row = (int)(e - (int64_t)col * n);
    Q[e] = (row == col) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = b - 1; j >= 0; --j) {
    const double t = tau[j];
    if (t == 0.0) continue;
    const double* vj = W + (int64_t)n * j;
    for (int l = j + warp; l < b; l += nw) {
      double* ql = Q + (int64_t)n * l;
      double dot = 0.0;
      for (int i = j + 1 + lane; i < n; i += 32) dot = fma(vj[i], ql[i], dot);
      dot = warp_sum(dot) + ql[j];
      const double w = t * dot;
      if (lane == 0) ql[j] -= w;
      for (int i = j + 1 + lane; i < n; i += 32) ql[i] = fma(-w, vj[i], ql[i]);
    }
    __syncthreads();
  }
  for (int l = warp; l < b; l += nw) {
    if (W[(int64_t)n * l + l] < 0.0) {
      double* ql = Q + (int64_t)n * l;
      for (int i = lane; i < n; i += 32) ql[i] = -ql[i];
    }
  }
  if (threadIdx.x == 0 && sh_bad) record_status(status, TKS_ENONFINITE);
}

}  // namespace

// ----------------------------------------------------------------------------- launchers
static int grid_for(int64_t work, int threads) {
  const int64_t g = (work + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

void launch_omega(const OmegaJob* jobs, int njobs, int64_t total_blocks, const Bases& bases,
                  uint64_t seed, cudaStream_t stream) {
  omega_kernel<<<grid_for(total_blocks, 256), 256, 0, stream>>>(jobs, njobs, total_blocks, bases, seed);
}

void launch_gemm_f64(const GemmJob* jobs, int njobs, int total_tiles, const Bases& bases,
                     cudaStream_t stream) {
  gemm_f64_kernel<<<total_tiles, 256, 0, stream>>>(jobs, njobs, bases);
}

void launch_splitk_reduce_f64(const GemmJob* jobs, int njobs, int64_t total_elems,
                              const Bases& bases, cudaStream_t stream) {
  splitk_reduce_f64_kernel<<<grid_for(total_elems, 256), 256, 0, stream>>>(jobs, njobs, total_elems,
                                                                          bases);
}

void launch_core_sketch_f64(const CoreSketchJob* jobs, int njobs, int64_t total, const Bases& bases,
                            cudaStream_t stream) {
  core_sketch_f64_kernel<<<grid_for(total, 128), 128, 0, stream>>>(jobs, njobs, total, bases);
}

void launch_qr_f64(const QrJob* jobs, int njobs, const Bases& bases, Status* status,
                   cudaStream_t stream) {
  qr_f64_kernel<<<njobs, 256, 0, stream>>>(jobs, bases, status);
}

}  // namespace tks

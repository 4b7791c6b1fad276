// Float64 small dense linear algebra of the ST-HOSVD truncation (Alg. 2 phase 2) for the TKS_FP64 and
// TKS_MIXED plans: the triangular factor R of each unfolding H_(n)^T by TSQR (Householder blocks held in
// registers) and a one-sided Jacobi SVD of R, whose right singular vectors are the left singular vectors
// of H_(n).  No Gram matrix is formed, so the kept subspaces carry float64 rounding relative to ||H||
// rather than ||H||^2 over the spectral gap.
//
// GB300 issues about two float64 FMAs per SM per clock (1/64 of the float32 rate), so both kernels are
// bound by the FP64 pipe, not by memory or latency: a column step of a 256-row TSQR block is about a
// thousand warp-level FMAs, against a few hundred cycles of reduction and barrier.
#include <cuda_runtime.h>

#include "fastdiv.cuh"
#include "kernels.h"

namespace tks {

namespace {

__device__ __forceinline__ void record_status_64(Status* st, int code) {
  if (st) atomicCAS(&st->code, 0, code);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of kN independent values with their butterflies interleaved.
template <int kN>
__device__ __forceinline__ void warp_sum_nd(double (&v)[kN]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < kN; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
}

// Step j of the register-resident Householder sweep: a_l -= tau v_j (v_j^T a_l) for every column
// l > j (l < ncols) this warp holds (column l lives in warp l % kWarps, slot l / kWarps).
template <int kRpl, int kSlots, int kWarps>
__device__ __forceinline__ void apply_reflector_d(double (&a)[kSlots][kRpl], const double (&vj)[kRpl], double tau,
                                                  int j, int ncols) {
  const int warp = threadIdx.x >> 5;
  if (tau == 0.0) return;
  double dot[kSlots];
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kWarps * sl;
    double d0 = 0.0, d1 = 0.0;
    if (l > j && l < ncols) {   // warp-uniform: finished and absent columns skip the products
#pragma unroll
      for (int u = 0; u + 1 < kRpl; u += 2) {
        d0 = fma(vj[u], a[sl][u], d0);
        d1 = fma(vj[u + 1], a[sl][u + 1], d1);
      }
      if (kRpl & 1) d0 = fma(vj[kRpl - 1], a[sl][kRpl - 1], d0);
    }
    dot[sl] = d0 + d1;
  }
  warp_sum_nd(dot);
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kWarps * sl;
    if (l > j && l < ncols) {
      const double w = tau * dot[sl];
#pragma unroll
      for (int u = 0; u < kRpl; ++u) a[sl][u] = fma(-w, vj[u], a[sl][u]);
    }
  }
}

// Forms the Householder reflector of column c (held by this warp: value a[u] at row lane + 32 u,
// m rows) that zeroes the rows below c, and publishes v = (0, .., 0, 1, x / (alpha - beta)) into
// v_out[0, vlen), tau = (beta - alpha) / beta and the diagonal entry beta of R.  A column whose
// rows below c are already zero gets tau = 0 and keeps its diagonal entry.  Returns false when the
// column norm is not finite.
template <int kRpl>
__device__ __forceinline__ bool reflector_publish_d(const double (&a)[kRpl], int c, int m, double* v_out, int vlen,
                                                    double* tau_out, double* rdiag) {
  const int lane = threadIdx.x & 31;
  double t2 = 0.0, alpha = 0.0;
#pragma unroll
  for (int u = 0; u < kRpl; ++u) {
    const int i = lane + 32 * u;
    if (i > c && i < m) t2 = fma(a[u], a[u], t2);
    if (i == c) alpha = a[u];
  }
  t2 = warp_sum_d(t2);
  alpha = __shfl_sync(0xffffffffu, alpha, c & 31);
  const double nrm = sqrt(fma(alpha, alpha, t2));
  const bool reflect = t2 > 0.0 && isfinite(nrm);
  const double beta = alpha >= 0.0 ? -nrm : nrm;
  const double tau = reflect ? (beta - alpha) / beta : 0.0;
  const double sc = reflect ? 1.0 / (alpha - beta) : 0.0;
#pragma unroll
  for (int u = 0; u < kRpl; ++u) {
    const int i = lane + 32 * u;
    if (i < vlen) v_out[i] = i < c ? 0.0 : (i == c ? 1.0 : (i < m ? sc * a[u] : 0.0));
  }
  if (lane == 0) {
    *tau_out = tau;
    rdiag[c] = reflect ? beta : alpha;
  }
  return isfinite(nrm);
}

// ----------------------------------------------------------------------------- TSQR block (float64)
// Householder QR of a rows x cols block of a float64 source read through a two-level row index
// (rows <= 32 kRpl, cols <= 16 kSlots); only the triangular factor is kept.  The block is staged
// through shared memory (coalesced along whichever index is contiguous in the source) and then
// lives in registers: column l in warp l % 16 (slot l / 16), lane L holds rows L + 32 u.  Each step j
// reads the published reflector v_j and tau_j, every warp updates its columns l > j, and the warp
// owning column j + 1 forms and publishes the next reflector: one barrier per column.
constexpr int kT64Threads = 512;
constexpr int kT64Warps = kT64Threads / 32;
constexpr int kT64LoadBatch = 8;

template <int kRpl, int kSlots>
__global__ void __launch_bounds__(kT64Threads, 1) tsqr_f64_kernel(const TsqrJob* __restrict__ jobs, Bases bases) {
  constexpr int kBlockRows = 32 * kRpl;
  extern __shared__ double smem_t64[];
  __shared__ double vbuf[2][kBlockRows];
  __shared__ double sh_tau[2];
  __shared__ double rdiag[kT64Warps * kSlots];
  __shared__ int64_t rowoff[kBlockRows];
  const TsqrJob& J = jobs[blockIdx.x];
  const int m = J.rows, b = J.cols;
  const int ld = m + 1;
  double* A = smem_t64;
  const double* src = at<double>(bases, J.src);
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const uint64_t i = (uint64_t)(J.row_begin + r), L0 = (uint64_t)J.L0;
    const uint64_t i1 = i / L0, i0 = i - i1 * L0;
    rowoff[r] = (int64_t)i0 * J.s0 + (int64_t)i1 * J.s1;
  }
  __syncthreads();
  const bool row_major = J.sc == 1;
  const int mb = m * b;   // <= 256 x 64 or 192 x 96, below 2^15
  const SmallDiv dq(row_major ? b : m);
  for (int e0 = 0; e0 < mb; e0 += kT64LoadBatch * kT64Threads) {
    double v[kT64LoadBatch];
    int dst[kT64LoadBatch];
#pragma unroll
    for (int u = 0; u < kT64LoadBatch; ++u) {
      const int e = e0 + u * kT64Threads + threadIdx.x;
      v[u] = 0.0;
      dst[u] = -1;
      if (e < mb) {
        const int q = dq.quo(e);
        const int r = row_major ? q : e - q * m, c = row_major ? e - q * b : q;
        v[u] = src[rowoff[r] + (int64_t)c * J.sc];
        dst[u] = r + ld * c;
      }
    }
#pragma unroll
    for (int u = 0; u < kT64LoadBatch; ++u)
      if (dst[u] >= 0) A[dst[u]] = v[u];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double a[kSlots][kRpl];
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kT64Warps * sl;
#pragma unroll
    for (int u = 0; u < kRpl; ++u) {
      const int i = lane + 32 * u;
      a[sl][u] = (l < b && i < m) ? A[i + ld * l] : 0.0;
    }
  }
  const int kmax = m < b ? m : b;
  if (warp == 0 && kmax > 0) reflector_publish_d(a[0], 0, m, vbuf[0], kBlockRows, &sh_tau[0], rdiag);
  __syncthreads();
  for (int j = 0; j < kmax; ++j) {
    const double tau = sh_tau[j & 1];
    double vj[kRpl];
#pragma unroll
    for (int u = 0; u < kRpl; ++u) vj[u] = vbuf[j & 1][lane + 32 * u];
    apply_reflector_d<kRpl, kSlots, kT64Warps>(a, vj, tau, j, b);
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
      const int l = warp + kT64Warps * sl;
      if (l == j + 1 && l < kmax)
        reflector_publish_d(a[sl], l, m, vbuf[(j + 1) & 1], kBlockRows, &sh_tau[(j + 1) & 1], rdiag);
    }
    __syncthreads();
  }
  // R: entries above the diagonal from the owner's registers, the diagonal from rdiag, zeros below
  // (and in rows at or beyond min(rows, cols))
  double* dst = at<double>(bases, J.dst);
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int c = warp + kT64Warps * sl;
    if (c < b) {
#pragma unroll
      for (int u = 0; u < kRpl; ++u) {
        const int r = lane + 32 * u;
        if (r < b) {
          double v = 0.0;
          if (r < kmax && r <= c) v = (r == c) ? rdiag[r] : a[sl][u];
          dst[(J.dst_row0 + r) + J.dst_ld * c] = v;
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------- Jacobi SVD (float64)
// One-sided (Hestenes) Jacobi on the columns of the b x b factor A = R with the round-robin ordering:
// each round rotates b/2 disjoint column pairs (kJ64Lanes lanes per pair, two rows per lane and
// chunk) until they are orthogonal; V accumulates the rotations, so that at convergence
// R V = U Sigma and the columns of V are the right singular vectors of R, i.e. the left singular
// vectors of H_(n).  Then: singular values = column norms, sorted; the rank rule of Alg. 2; P = the
// leading columns of V, sign-fixed (largest-magnitude entry positive), zero-padded to rmax.
constexpr int kJ64Sweeps = 40;
constexpr int kJ64Lanes = 8;
constexpr int kJ64Threads = kJ64Lanes * (TKS_MAX_BASIS / 2);   // 384
constexpr int kJ64Chunks = (TKS_MAX_BASIS + 2 * kJ64Lanes - 1) / (2 * kJ64Lanes);   // 2-row chunks per lane

__device__ double block_sum_d(double v, double* red) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];   // fixed order
  return s;
}

__global__ void __launch_bounds__(kJ64Threads) svd_jacobi_f64_kernel(const SvdJob* __restrict__ jobs, Bases bases,
                                                                   Status* status) {
  extern __shared__ double sm64[];
  const SvdJob& J = jobs[blockIdx.x];
  const int b = J.b;
  const int m = b + (b & 1);
  const int ld = (m + 1) & ~1;   // columns start 16-byte aligned; rows in [b, ld) stay zero
  double* A = sm64;
  double* V = A + m * ld;
  double* nrm = V + m * ld;
  int* order = reinterpret_cast<int*>(nrm + m);
  __shared__ int sh_rot, sh_rank;
  __shared__ double red[32];
  __shared__ double sh_noise2;
  const double* Rg = at<double>(bases, J.R);
  for (int e = threadIdx.x; e < m * ld; e += blockDim.x) {
    const int r = e % ld, c = e / ld;
    A[e] = (r < b && c < b) ? Rg[r + c * b] : 0.0;
    V[e] = (r == c) ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) sh_noise2 = 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // rotate while |a_p . a_q| > b eps ||a_p|| ||a_q||, except for columns at the float64 noise floor
  // (norm <= 8 eps times the largest column norm): their couplings are rounding noise
  const double eps = 1.1102230246251565e-16;
  const double thr = (double)b * eps;
  for (int c = warp; c < b; c += nw) {
    double s2 = 0.0;
    for (int i = lane; i < b; i += 32) s2 = fma(A[i + c * ld], A[i + c * ld], s2);
    s2 = warp_sum_d(s2);
    // non-negative doubles order like their bit patterns
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(&sh_noise2), (unsigned long long)__double_as_longlong(s2));
  }
  __syncthreads();
  const double noise2 = sh_noise2 * (8.0 * eps) * (8.0 * eps);
  const int sub = lane % kJ64Lanes;
  const int k = threadIdx.x / kJ64Lanes;
  const int pairs = m / 2;
  int sweep = 0;
  for (; sweep < kJ64Sweeps; ++sweep) {
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
      double* ap = A + p * ld;
      double* aq = A + q * ld;
      double2 x[kJ64Chunks], y[kJ64Chunks];
      double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
      for (int u = 0; u < kJ64Chunks; ++u) {
        const int i = 2 * (sub + kJ64Lanes * u);
        const bool in = valid && i < b;
        x[u] = in ? *reinterpret_cast<const double2*>(ap + i) : make_double2(0.0, 0.0);
        y[u] = in ? *reinterpret_cast<const double2*>(aq + i) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int u = 0; u < kJ64Chunks; ++u) {
        al = fma(x[u].x, x[u].x, fma(x[u].y, x[u].y, al));
        be = fma(y[u].x, y[u].x, fma(y[u].y, y[u].y, be));
        ga = fma(x[u].x, y[u].x, fma(x[u].y, y[u].y, ga));
      }
#pragma unroll
      for (int o = kJ64Lanes / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o, kJ64Lanes);
        be += __shfl_xor_sync(0xffffffffu, be, o, kJ64Lanes);
        ga += __shfl_xor_sync(0xffffffffu, ga, o, kJ64Lanes);
      }
      if (valid && fabs(ga) > thr * sqrt(al * be) && ga != 0.0 && fmin(al, be) > noise2) {
        // rotation that zeroes the (p, q) entry of A^T A (Golub & Van Loan, symmetric 2 x 2 Schur)
        const double zeta = (be - al) / (2.0 * ga);
        const double az = fabs(zeta);
        const double tm = az > 1e150 ? 0.5 / az : 1.0 / (az + sqrt(fma(az, az, 1.0)));
        const double t = copysign(tm, zeta);
        const double c = 1.0 / sqrt(fma(t, t, 1.0));
        const double s = c * t;
        double* vp = V + p * ld;
        double* vq = V + q * ld;
#pragma unroll
        for (int u = 0; u < kJ64Chunks; ++u) {
          const int i = 2 * (sub + kJ64Lanes * u);
          if (i < b) {
            const double2 a0 = x[u], b0 = y[u];
            *reinterpret_cast<double2*>(ap + i) = make_double2(c * a0.x - s * b0.x, c * a0.y - s * b0.y);
            *reinterpret_cast<double2*>(aq + i) = make_double2(s * a0.x + c * b0.x, s * a0.y + c * b0.y);
            const double2 vx = *reinterpret_cast<const double2*>(vp + i);
            const double2 vy = *reinterpret_cast<const double2*>(vq + i);
            *reinterpret_cast<double2*>(vp + i) = make_double2(c * vx.x - s * vy.x, c * vx.y - s * vy.y);
            *reinterpret_cast<double2*>(vq + i) = make_double2(s * vx.x + c * vy.x, s * vx.y + c * vy.y);
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
  // squared singular values = squared column norms; order them by decreasing value
  for (int c = warp; c < b; c += nw) {
    double s = 0.0;
    for (int i = lane; i < b; i += 32) s = fma(A[i + c * ld], A[i + c * ld], s);
    s = warp_sum_d(s);
    if (lane == 0) nrm[c] = s;
  }
  __syncthreads();
  double tot = 0.0;
  {
    double part = 0.0;
    for (int i = threadIdx.x; i < b; i += blockDim.x) part += nrm[i];
    tot = block_sum_d(part, red);
  }
  // thread i places column i at its rank (ties by index; a NaN counts as -1 so the ranks always
  // form a permutation)
  if ((int)threadIdx.x < b) {
    const int i = threadIdx.x;
    const double ni = nrm[i] == nrm[i] ? nrm[i] : -1.0;
    int rk = 0;
    for (int j = 0; j < b; ++j) {
      const double nj = nrm[j] == nrm[j] ? nrm[j] : -1.0;
      rk += (nj > ni || (nj == ni && j < i)) ? 1 : 0;
    }
    order[rk] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double* sv = at<double>(bases, J.sv);
    for (int i = 0; i < b; ++i) sv[i] = sqrt(fmax(nrm[order[i]], 0.0));
    double* theta = at<double>(bases, J.theta);
    if (J.first_mode) *theta = J.tol * J.tol * tot / J.order;
    int r = J.rmax;
    if (J.tol > 0.0) {
      // r = min{r >= 1 : sum_{j > r} sigma_j^2 <= theta} (Alg. 2), capped by rmax
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
    if (!isfinite(tot)) record_status_64(status, TKS_ENONFINITE);
    if (sweep >= kJ64Sweeps) record_status_64(status, TKS_ENOCONV);
  }
  __syncthreads();
  const int r = sh_rank;
  double* P = at<double>(bases, J.P);
  for (int t = warp; t < J.rmax; t += nw) {
    if (t >= r) {
      for (int i = lane; i < b; i += 32) P[i + (int64_t)t * b] = 0.0;
      continue;
    }
    const int src = order[t];
    double best = 0.0;
    for (int i = lane; i < b; i += 32) {
      const double v = V[i + src * ld];
      if (fabs(v) > fabs(best)) best = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, best, o);
      if (fabs(other) > fabs(best) || (fabs(other) == fabs(best) && other > best)) best = other;
    }
    const double sgn = (best < 0.0) ? -1.0 : 1.0;
    for (int i = lane; i < b; i += 32) P[i + (int64_t)t * b] = sgn * V[i + src * ld];
  }
}

size_t svd64_smem(int bmax) {
  const int m = bmax + (bmax & 1), ld = (m + 1) & ~1;
  return (size_t)2 * m * ld * sizeof(double) + (size_t)m * sizeof(double) + (size_t)m * sizeof(int);
}

size_t tsqr64_smem(int rows, int cols) { return (size_t)(rows + 1) * cols * sizeof(double); }

}  // namespace

// At least twice the columns, so that every TSQR level shrinks the stack of factors.
int tsqr64_block_rows(int max_cols) { return max_cols <= 4 * kT64Warps ? 256 : 192; }

cudaError_t prepare_la64(int bmax) {
  cudaError_t e = cudaFuncSetAttribute(svd_jacobi_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)svd64_smem(bmax));
  if (e != cudaSuccess) return e;
  const void* kernels[] = {reinterpret_cast<const void*>(tsqr_f64_kernel<8, 2>),
                           reinterpret_cast<const void*>(tsqr_f64_kernel<8, 3>),
                           reinterpret_cast<const void*>(tsqr_f64_kernel<8, 4>),
                           reinterpret_cast<const void*>(tsqr_f64_kernel<6, 6>)};
  for (const void* k : kernels) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsqr64_smem(256, 64));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void launch_tsqr_f64(const TsqrJob* jobs, int njobs, int max_cols, const Bases& bases, cudaStream_t stream) {
  // columns per warp: the smallest instantiation that covers max_cols; 256-row blocks up to 64
  // columns, 192-row blocks beyond (the register tile stays at 32 or 36 doubles per thread)
  if (max_cols <= 2 * kT64Warps) {
    tsqr_f64_kernel<8, 2><<<njobs, kT64Threads, tsqr64_smem(256, 2 * kT64Warps), stream>>>(jobs, bases);
  } else if (max_cols <= 3 * kT64Warps) {
    tsqr_f64_kernel<8, 3><<<njobs, kT64Threads, tsqr64_smem(256, 3 * kT64Warps), stream>>>(jobs, bases);
  } else if (max_cols <= 4 * kT64Warps) {
    tsqr_f64_kernel<8, 4><<<njobs, kT64Threads, tsqr64_smem(256, 4 * kT64Warps), stream>>>(jobs, bases);
  } else {
    tsqr_f64_kernel<6, 6><<<njobs, kT64Threads, tsqr64_smem(192, 6 * kT64Warps), stream>>>(jobs, bases);
  }
}

void launch_svd_f64(const SvdJob* jobs, int njobs, int bmax, const Bases& bases, Status* status,
                    cudaStream_t stream) {
  const int pairs = (bmax + 1) / 2;
  const int threads = ((pairs * kJ64Lanes + 31) / 32) * 32;
  svd_jacobi_f64_kernel<<<njobs, threads, svd64_smem(bmax), stream>>>(jobs, bases, status);
}

}  // namespace tks

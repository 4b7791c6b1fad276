// Effective subrank heuristic (Alg. 5, Sec. 3.2) in float64.
//
// Per (problem, mode n):  V_n = [w_1 U_1^(n), ..., w_K U_K^(n)] with w_k = ||alpha_k G_k||_F, the
// Gram matrix of V_n, its eigenvalues (clamped at zero, descending), the threshold
// tau = eps^2 / d * sum_j lambda_j and rank = min{r >= 1 : sum_{j > r} lambda_j <= tau}.
//
// Kernels:
//   subrank_weight_kernel  one CTA per term: ||G_k||_F by a fixed-order block reduction, written
//                          as the weight of each of the term's columns in every mode.
//   gram_f64_kernel        64 x 64 float64 tiles of the lower triangle of V^T V (R <= n) or V V^T
//                          (n < R; same nonzero eigenvalues, smaller matrix), mirrored.
//   tridiag_f64_kernel     one CTA per matrix: Householder reduction to tridiagonal form on the
//                          lower triangle only: per step the pending rank-2 update of the previous
//                          step (2 FMAs per stored element) and the symmetric product p = A v (each
//                          stored element feeds two rows), 2 m^3 / 3 FMAs in all instead of m^3.
//   subrank_eig_kernel     one CTA per matrix: the tridiagonal matrix's eigenvalues by bisection
//                          with division-free Sturm counts (one eigenvalue per thread), rank rule,
//                          ell = rank + p.
// GB300 issues about two FP64 FMAs per SM per clock, so every kernel here is bound by FP64 issue;
// the matrices (m <= 2048) stay in global memory and L2.
#include <cuda_runtime.h>

#include "bf16.cuh"
#include "kernels.h"

namespace tks {

namespace {

__device__ __forceinline__ void record_status(Status* st, int code) {
  if (st) atomicCAS(&st->code, 0, code);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block in a fixed order (deterministic); every thread gets the result.
__device__ double block_sum_d(double v, double* red) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

__device__ double block_max_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s = fmax(s, red[w]);
  return s;
}

// ----------------------------------------------------------------------------- term weights
constexpr int kWeightThreads = 256;

__global__ void __launch_bounds__(kWeightThreads) subrank_weight_kernel(const WeightJob* __restrict__ jobs,
                                                                        Bases bases) {
  __shared__ double red[32];
  const WeightJob& J = jobs[blockIdx.x];
  double part = 0.0;
  if (J.type == T_BF16) {
    const uint16_t* g = at<uint16_t>(bases, J.core);
    for (int64_t e = threadIdx.x; e < J.count; e += kWeightThreads) {
      const double x = (double)bf16_float(g[e]);
      part = fma(x, x, part);
    }
  } else {
    const double* g = at<double>(bases, J.core);
    for (int64_t e = threadIdx.x; e < J.count; e += kWeightThreads) part = fma(g[e], g[e], part);
  }
  const double w = fabs(J.alpha) * sqrt(block_sum_d(part, red));
  for (int m = 0; m < J.d; ++m) {
    double* wc = at<double>(bases, J.wcol[m]);
    for (int i = threadIdx.x; i < J.r[m]; i += kWeightThreads) wc[i] = w;
  }
}

// ----------------------------------------------------------------------------- Gram tiles
constexpr int kGT = 64;        // output tile
constexpr int kGK = 16;        // contraction chunk
constexpr int kGThreads = 256; // 16 x 16 threads, 4 x 4 outputs each
constexpr int kGPad = kGT + 2;

__device__ __forceinline__ double load_typed(const char* base, int32_t type, int64_t idx) {
  return type == T_BF16 ? (double)bf16_float(reinterpret_cast<const uint16_t*>(base)[idx])
                        : reinterpret_cast<const double*>(base)[idx];
}

__global__ void __launch_bounds__(kGThreads) gram_f64_kernel(const GramJob* __restrict__ jobs, int njobs,
                                                             Bases bases) {
  __shared__ double As[kGK][kGPad];
  __shared__ double Bs[kGK][kGPad];
  const int lo = tile_job(jobs, njobs, (int)blockIdx.x);
  const GramJob& J = jobs[lo];
  const int t = (int)blockIdx.x - J.tile_begin;
  int ti = 0;
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int row0 = ti * kGT, col0 = tj * kGT, m = J.m;
  const int64_t n = J.n;
  const int64_t kc = J.aat ? (int64_t)J.R : n;   // contraction length
  const char* U = at<char>(bases, J.U);
  const double* wcol = at<double>(bases, J.wcol);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = 0; k0 < kc; k0 += kGK) {
    if (!J.aat) {
      // X(a, i) = U[i + n a]: tile column a of U, contraction over the rows i
      for (int e = threadIdx.x; e < kGK * kGT; e += kGThreads) {
        const int kk = e % kGK, a = e / kGK;
        const int64_t i = k0 + kk;
        const int ra = row0 + a, cb = col0 + a;
        As[kk][a] = (i < kc && ra < m) ? load_typed(U, J.type, i + n * ra) : 0.0;
        Bs[kk][a] = (i < kc && cb < m) ? load_typed(U, J.type, i + n * cb) : 0.0;
      }
    } else {
      // X(i, c) = w_c U[i + n c]: tile row i of U, contraction over the columns c
      for (int e = threadIdx.x; e < kGK * kGT; e += kGThreads) {
        const int a = e % kGT, kk = e / kGT;
        const int64_t c = k0 + kk;
        const int ra = row0 + a, cb = col0 + a;
        const double w = c < kc ? wcol[c] : 0.0;
        As[kk][a] = (c < kc && ra < m) ? w * load_typed(U, J.type, ra + n * c) : 0.0;
        Bs[kk][a] = (c < kc && cb < m) ? w * load_typed(U, J.type, cb + n * c) : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = As[kk][ty * 4 + i];
        bv[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* B = at<double>(bases, J.B);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty * 4 + i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx * 4 + j;
      if (c >= m || c > r) continue;
      const double v = J.aat ? acc[i][j] : wcol[r] * wcol[c] * acc[i][j];
      B[r + (int64_t)m * c] = v;
      B[c + (int64_t)m * r] = v;
    }
  }
}

// ----------------------------------------------------------------------------- tridiagonalization
constexpr int kTriThreads = 512;

// Rows are owned by absolute index: thread t holds rows t + kTriThreads q, q < kRows, so the
// previous step's v_i, w_i for its rows stay in registers from one step to the next.
template <int kRows>
__global__ void __launch_bounds__(kTriThreads, 1) tridiag_f64_kernel(const SubrankJob* __restrict__ jobs,
                                                                    Bases bases, Status* status) {
  extern __shared__ double tsm[];
  __shared__ double red[32];
  const SubrankJob& J = jobs[blockIdx.x];
  const int m = J.m;
  double* A = at<double>(bases, J.B);
  double* dg = at<double>(bases, J.d);
  double* eg = at<double>(bases, J.e);
  double* vc = tsm;            // v of this step (rows k+1..m-1, v_{k+1} = 1)
  double* vp = tsm + m;        // v of the previous step
  double* wc = tsm + 2 * m;    // w of this step
  double* wp = tsm + 3 * m;    // w of the previous step
  const int tid = threadIdx.x;
  double vpr[kRows], wpr[kRows], p[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) vpr[q] = wpr[q] = 0.0;
  bool have_prev = false;
  bool bad = false;
  bool stopped = false;
  int executed = m > 1 ? m - 1 : 0;
  double delta = 0.0;
  for (int k = 0; k + 1 < m; ++k) {
    double* colk = A + (int64_t)m * k;
    // column k, rows k..m-1: apply the previous step's update
    if (have_prev) {
      const double vk = vp[k], wk = wp[k];
      for (int i = k + tid; i < m; i += kTriThreads) colk[i] = fma(-vp[i], wk, fma(-wp[i], vk, colk[i]));
    }
    __syncthreads();
    // Early end: the trailing block C = A[k:, k:] of the (positive semidefinite) Gram matrix, with
    // the pending update, has sum |c_ii| <= delta.  Replacing C by zero moves the eigenvalues by a
    // total of at most trace(C) (nuclear norm of a semidefinite perturbation), so every sum of the
    // rank rule changes by at most delta = min(m u trace(B), 2^-10 tau): the rounding level of the
    // reduction, and far below the threshold.  This skips the numerically zero part of a
    // rank-deficient Gram matrix.
    {
      double part = 0.0;
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        const int i = tid + q * kTriThreads;
        if (i == k) part += fabs(colk[k]);
        else if (i > k && i < m)
          part += fabs(have_prev ? fma(-2.0 * vpr[q], wpr[q], A[i + (int64_t)m * i]) : A[i + (int64_t)m * i]);
      }
      const double trail = block_sum_d(part, red);
      if (k == 0) delta = fmin(m * 0x1p-53 * trail, 0x1p-10 * J.eps * J.eps / J.order * trail);
      if (trail <= delta) {
        for (int i = k + tid; i < m; i += kTriThreads) {
          dg[i] = 0.0;
          eg[i] = 0.0;
        }
        stopped = true;
        executed = k;
        break;
      }
    }
    // Householder reflector H = I - tau v v^T with H x = beta e_1, x = A[k+1:m, k]; the norm is
    // taken of x scaled by a power of two near 1 / max |x_i| (no underflow or overflow of x_i^2)
    double amax = 0.0;
    for (int i = k + 1 + tid; i < m; i += kTriThreads) amax = fmax(amax, fabs(colk[i]));
    amax = block_max_d(amax, red);
    const double alpha = colk[k + 1];
    double tau = 0.0, beta = alpha, scale = 0.0;
    if (amax > 0.0 && isfinite(amax)) {
      const double sc = ldexp(1.0, -ilogb(amax));
      double part = 0.0;
      for (int i = k + 2 + tid; i < m; i += kTriThreads) {
        const double x = colk[i] * sc;
        part = fma(x, x, part);
      }
      const double sigma = block_sum_d(part, red);
      if (sigma > 0.0) {
        const double as = alpha * sc;
        const double mu = sqrt(fma(as, as, sigma)) / sc;
        beta = alpha <= 0.0 ? mu : -mu;
        tau = (beta - alpha) / beta;
        scale = 1.0 / (alpha - beta);
      }
    }
    if (!isfinite(amax)) bad = true;
    if (tid == 0) {
      dg[k] = colk[k];
      eg[k] = beta;
    }
    for (int i = k + 1 + tid; i < m; i += kTriThreads) vc[i] = i == k + 1 ? 1.0 : colk[i] * scale;
    __syncthreads();
    // Trailing block rows/cols k+1..m-1, lower triangle only (the upper one is never read).
    // Pass 1: the pending rank-2 update of step k-1, a_ij -= v_i w_j + w_i v_j for j <= i.
    if (have_prev) {
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        const int i = tid + q * kTriThreads;
        if (i > k && i < m) {
          double* row = A + i;
          const double vi = vpr[q], wi = wpr[q];
          int j = k + 1;
          for (; j + 4 <= i + 1; j += 4) {
            double x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = row[(int64_t)m * (j + u)];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              row[(int64_t)m * (j + u)] = fma(-vi, wp[j + u], fma(-wi, vp[j + u], x[u]));
          }
          for (; j <= i; ++j) row[(int64_t)m * j] = fma(-vi, wp[j], fma(-wi, vp[j], row[(int64_t)m * j]));
        }
      }
      __syncthreads();
    }
    // Pass 2: p = A v from the lower triangle: row i left of the diagonal (coalesced over the
    // threads) and column i below it (contiguous for each thread).  Every thread reads m - k - 1
    // elements per row it owns, and each stored element feeds two rows of p.
#pragma unroll
    for (int q = 0; q < kRows; ++q) p[q] = 0.0;
    if (tau != 0.0) {
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        const int i = tid + q * kTriThreads;
        if (i > k && i < m) {
          const double* row = A + i;
          double s0 = 0.0, s1 = 0.0;
          int j = k + 1;
          for (; j + 4 <= i + 1; j += 4) {
            double x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = row[(int64_t)m * (j + u)];
            s0 = fma(x[0], vc[j], s0);
            s1 = fma(x[1], vc[j + 1], s1);
            s0 = fma(x[2], vc[j + 2], s0);
            s1 = fma(x[3], vc[j + 3], s1);
          }
          for (; j <= i; ++j) s0 = fma(row[(int64_t)m * j], vc[j], s0);
          const double* col = A + (int64_t)m * i;
          j = i + 1;
          for (; j + 4 <= m; j += 4) {
            double x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = col[j + u];
            s0 = fma(x[0], vc[j], s0);
            s1 = fma(x[1], vc[j + 1], s1);
            s0 = fma(x[2], vc[j + 2], s0);
            s1 = fma(x[3], vc[j + 3], s1);
          }
          for (; j < m; ++j) s1 = fma(col[j], vc[j], s1);
          p[q] = s0 + s1;
        }
      }
    }
    // w = tau A v - (tau^2 / 2)(v^T A v) v
    double pv = 0.0;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      const int i = tid + q * kTriThreads;
      if (i > k && i < m) pv = fma(p[q], vc[i], pv);
    }
    const double vav = block_sum_d(pv, red);
    const double half = 0.5 * tau * tau * vav;
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      const int i = tid + q * kTriThreads;
      if (i > k && i < m) {
        const double w = fma(tau, p[q], -half * vc[i]);
        wc[i] = w;
        vpr[q] = vc[i];
        wpr[q] = w;
      }
    }
    have_prev = tau != 0.0;
    double* t0 = vp; vp = vc; vc = t0;
    double* t1 = wp; wp = wc; wc = t1;
    __syncthreads();
  }
  if (tid == 0 && !stopped) {
    dg[m - 1] = A[(int64_t)m * m - 1];
    eg[m - 1] = 0.0;
    if (!isfinite(dg[m - 1])) bad = true;
  }
  if (tid == 0 && J.steps) *J.steps = executed;
  if (bad) record_status(status, TKS_ENONFINITE);
}

// ----------------------------------------------------------------------------- eigenvalues + rule
constexpr int kEigThreads = 256;
constexpr int kBisectMaxIter = 64;

__device__ __forceinline__ int sign_bit(double v) {
  return (int)((unsigned long long)__double_as_longlong(v) >> 63);
}
__device__ __forceinline__ int exponent_bits(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
}

// Number of eigenvalues smaller than x of the symmetric tridiagonal matrix with diagonal d and
// squared off-diagonals e2 (n x n): the sign changes of the Sturm sequence of its leading
// principal minors, p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2} with p_{-1} = 1 (Givens' bisection,
// Wilkinson, The Algebraic Eigenvalue Problem, Ch. 5).  A zero p_i takes the sign opposite to
// p_{i-1} (the limit of a small negative pivot).  The pair (p_{i-1}, p_i) is rescaled by 2^-+256
// when p_i leaves [2^-256, 2^256], so nothing overflows or underflows; signs and exponents are
// read from the bits.  Three float64 operations per row, no division: on GB300 a division is a
// long chain of dependent float64 operations.
__device__ int sturm_count(const double* d, const double* e2, int n, double x) {
  double p0 = 1.0, p1 = d[0] - x;
  int sp = (__double_as_longlong(p1) << 1) == 0 ? 1 : sign_bit(p1);
  int cnt = sp;
  for (int i = 1; i < n; ++i) {
    double p2 = fma(d[i] - x, p1, -e2[i - 1] * p0);
    const long long bits = __double_as_longlong(p2);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex > 1023 + 256) {
      p2 *= 0x1p-256;
      p1 *= 0x1p-256;
    } else if (ex < 1023 - 256 && (bits << 1) != 0 && exponent_bits(p1) < 1023 + 256) {
      p2 *= 0x1p+256;
      p1 *= 0x1p+256;
    }
    const int s2 = (bits << 1) == 0 ? 1 - sp : (int)((unsigned long long)bits >> 63);
    cnt += s2 != sp;
    sp = s2;
    p0 = p1;
    p1 = p2;
  }
  return cnt;
}

__device__ double block_min_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = red[0];
  for (int w = 1; w < nw; ++w) s = fmin(s, red[w]);
  return s;
}

// Eigenvalues of the tridiagonal matrix by bisection, one eigenvalue per thread (every thread
// runs the same Sturm recurrence on a different shift, so the block is throughput-bound rather
// than bound by the latency of one long sequential chain), then the rank rule.  Rows after the
// last nonzero diagonal or off-diagonal entry form an exact zero block (the early end of the
// reduction) and contribute zero eigenvalues without bisection.
__global__ void __launch_bounds__(kEigThreads) subrank_eig_kernel(const SubrankJob* __restrict__ jobs, Bases bases,
                                                                  Status* status) {
  extern __shared__ double esm[];
  __shared__ double red[32];
  __shared__ int sh_last;
  const SubrankJob& J = jobs[blockIdx.x];
  const int m = J.m;
  double* d = esm;
  double* e2 = esm + m;
  double* lam = esm + 2 * m;
  const double* dg = at<double>(bases, J.d);
  const double* eg = at<double>(bases, J.e);
  if (threadIdx.x == 0) sh_last = -1;
  __syncthreads();
  // active size, infinity norm (Gershgorin) of the active block
  double tn = 0.0;
  for (int i = threadIdx.x; i < m; i += kEigThreads) {
    const double di = dg[i], ei = i + 1 < m ? eg[i] : 0.0, em = i > 0 ? eg[i - 1] : 0.0;
    if (di != 0.0 || em != 0.0) atomicMax(&sh_last, i);
    tn = fmax(tn, fabs(di) + fabs(ei) + fabs(em));
  }
  tn = block_max_d(tn, red);
  const int n = sh_last + 1;
  const bool finite = isfinite(tn);
  double sc = 1.0;
  if (tn > 0.0 && finite) sc = ldexp(1.0, -ilogb(tn));
  double glo = 0.0, ghi = 0.0;
  for (int i = threadIdx.x; i < n; i += kEigThreads) {
    const double di = dg[i] * sc, ei = i + 1 < n ? eg[i] * sc : 0.0, em = i > 0 ? eg[i - 1] * sc : 0.0;
    d[i] = di;
    e2[i] = ei * ei;
    glo = fmin(glo, di - fabs(ei) - fabs(em));
    ghi = fmax(ghi, di + fabs(ei) + fabs(em));
  }
  glo = block_min_d(glo, red);
  ghi = block_max_d(ghi, red);   // ends with a barrier: d, e2 are complete
  if (finite) {
    const double tol = 0x1p-50 * fmax(fabs(glo), fabs(ghi));
    for (int j = threadIdx.x; j < n; j += kEigThreads) {
      double lo = glo, hi = ghi;
      for (int it = 0; it < kBisectMaxIter && hi - lo > tol; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(d, e2, n, mid) > j) hi = mid; else lo = mid;
      }
      lam[j] = 0.5 * (lo + hi) / sc;   // ascending in j
    }
  }
  __syncthreads();
  // all m eigenvalues in descending order: the active ones with the m - n zeros merged in
  int npos = 0;
  for (int j = threadIdx.x; j < n; j += kEigThreads) npos += finite && lam[j] > 0.0;
  npos = (int)block_sum_d((double)npos, red);
  double* ev = at<double>(bases, J.ev);
  for (int t = threadIdx.x; t < m; t += kEigThreads) {
    double v;
    if (!finite) v = tn;
    else if (t < npos) v = lam[n - 1 - t];
    else if (t < npos + (m - n)) v = 0.0;
    else v = lam[n - 1 - (t - (m - n))];
    ev[t] = v;
  }
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int j = 0; j < n; ++j) total += finite ? fmax(lam[j], 0.0) : 0.0;
    const double tau = J.eps * J.eps / J.order * total;
    // the largest c <= m - 1 whose c smallest eigenvalues sum to at most tau; rank = m - c.
    // The m - n zeros (and the clamped negatives) come first in ascending order.
    double tail = 0.0;
    int c = 0;
    while (c < m - 1) {
      // c-th smallest: first the active eigenvalues <= 0 and the zero block (all clamp to 0)
      const int nonpos = m - npos;
      const double v = c < nonpos ? 0.0 : lam[n - npos + (c - nonpos)];
      const double next = tail + v;
      if (!(next <= tau)) break;
      tail = next;
      ++c;
    }
    const int rank = m - c;
    *at<int32_t>(bases, J.rank) = rank;
    *at<int32_t>(bases, J.ell) = rank + J.p;
    if (!finite) record_status(status, TKS_ENONFINITE);
  }
}

}  // namespace

void launch_subrank_weights(const WeightJob* jobs, int njobs, const Bases& bases, cudaStream_t stream) {
  subrank_weight_kernel<<<njobs, kWeightThreads, 0, stream>>>(jobs, bases);
}

void launch_gram_f64(const GramJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream) {
  gram_f64_kernel<<<total_tiles, kGThreads, 0, stream>>>(jobs, njobs, bases);
}

constexpr size_t kTriSmem = 4 * kSubrankMaxDim * sizeof(double);
constexpr size_t kEigSmem = 3 * kSubrankMaxDim * sizeof(double);

cudaError_t prepare_subrank() {
  cudaError_t e = cudaFuncSetAttribute(tridiag_f64_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tridiag_f64_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tridiag_f64_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTriSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(subrank_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmem);
  return e;
}

// max_m: the largest matrix of the launch (picks the rows each thread owns)
void launch_tridiag_f64(const SubrankJob* jobs, int njobs, int max_m, const Bases& bases, Status* status,
                        cudaStream_t stream) {
  const size_t smem = 4 * (size_t)max_m * sizeof(double);
  if (max_m <= kTriThreads)
    tridiag_f64_kernel<1><<<njobs, kTriThreads, smem, stream>>>(jobs, bases, status);
  else if (max_m <= 2 * kTriThreads)
    tridiag_f64_kernel<2><<<njobs, kTriThreads, smem, stream>>>(jobs, bases, status);
  else
    tridiag_f64_kernel<4><<<njobs, kTriThreads, smem, stream>>>(jobs, bases, status);
}

void launch_subrank_eig(const SubrankJob* jobs, int njobs, int max_m, const Bases& bases, Status* status,
                        cudaStream_t stream) {
  subrank_eig_kernel<<<njobs, kEigThreads, 3 * (size_t)max_m * sizeof(double), stream>>>(jobs, bases, status);
}

}  // namespace tks

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

#include <algorithm>

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

// Sums over the 32 lanes of kN (1, 2, 4 or 8) per-lane values; returns, in every lane, the total of
// value s(lane), where s(lane) collects the lane bits 16, 8, ... of the first log2(kN) levels (see
// slot_lane).  A transposed butterfly: at each of those levels a lane keeps half of its values and
// sends the other half, so the warp spends kN - 1 + 5 - log2(kN) additions per lane instead of 5 kN.
template <int kN>
__device__ __forceinline__ double warp_sum_transposed(double (&v)[kN]) {
  const int lane = threadIdx.x & 31;
  int o = 16;
#pragma unroll
  for (int h = kN / 2; h >= 1; h /= 2, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double send = up ? v[i] : v[i + h];
      const double keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  double r = v[0];
  for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// A lane that holds the total of value s after warp_sum_transposed<kN>.
template <int kN>
__device__ __forceinline__ int slot_lane(int s) {
  int lane = 0, o = 16;
#pragma unroll
  for (int h = kN / 2; h >= 1; h /= 2, o >>= 1)
    if (s & h) lane |= o;
  return lane;
}

// Step j of the register-resident Householder sweep: a_l -= tau v_j (v_j^T a_l) for every column
// l > j (l < ncols) this warp holds (column l lives in warp l % kWarps, slot l / kWarps).  Row slots
// u whose bit in umask is clear hold only rows where v_j is zero and are skipped.
template <int kRpl, int kSlots, int kWarps>
__device__ __forceinline__ void apply_reflector_d(double (&a)[kSlots][kRpl], const double (&vj)[kRpl], double tau,
                                                  int j, int ncols, unsigned umask) {
  const int warp = threadIdx.x >> 5;
  if (tau == 0.0) return;
  constexpr int kP = kSlots <= 1 ? 1 : kSlots <= 2 ? 2 : kSlots <= 4 ? 4 : 8;
  double dot[kP];
#pragma unroll
  for (int sl = 0; sl < kP; ++sl) {
    dot[sl] = 0.0;
    const int l = warp + kWarps * sl;
    if (sl < kSlots && l > j && l < ncols) {   // warp-uniform: finished and absent columns skip the products
      double d = 0.0;
#pragma unroll
      for (int u = 0; u < kRpl; ++u)
        if ((umask >> u) & 1u) d = fma(vj[u], a[sl < kSlots ? sl : 0][u], d);
      dot[sl] = d;
    }
  }
  // each lane scales the total it holds; the owner lanes broadcast w = tau v_j^T a_l
  const double w_own = tau * warp_sum_transposed<kP>(dot);
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    const int l = warp + kWarps * sl;
    const double w = __shfl_sync(0xffffffffu, w_own, slot_lane<kP>(sl));
    if (l > j && l < ncols) {
#pragma unroll
      for (int u = 0; u < kRpl; ++u)
        if ((umask >> u) & 1u) a[sl][u] = fma(-w, vj[u], a[sl][u]);
    }
  }
}

// 2^-e for the exponent e of x > 0 (x 2^-e in [1, 2)), or 0 when x is zero, subnormal, not finite
// or 2^-e is not a normal double; from the exponent bits, without a division.
__device__ __forceinline__ double pow2_inverse(double x) {
  const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return (ex >= 1 && ex <= 2045) ? __longlong_as_double((long long)(2046 - ex) << 52) : 0.0;
}

// 1 / sqrt(z) and 1 / x for normal z, x > 0 in float64 by Newton's method from a float32 estimate:
// the argument is scaled by a power of two into float32 range (an even power for the square root),
// and each Newton step squares the relative error (2^-22 -> 2^-44 -> below float64 rounding).  Far
// shorter dependent chains than a float64 division or square root, which matters where one thread's
// result gates a whole block (a Householder reflector per column).
__device__ __forceinline__ double rsqrt_newton(double z) {
  const int ex = (int)((__double_as_longlong(z) >> 52) & 0x7ff) - 1023;
  const int k = ex >> 1;                                     // z = z1 4^k, z1 in [1, 4)
  const double down = __longlong_as_double((long long)(1023 - 2 * k) << 52);
  const double up = __longlong_as_double((long long)(1023 - k) << 52);
  const double z1 = z * down, h = 0.5 * z1;
  double y = (double)rsqrtf((float)z1);
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y * up;
}
__device__ __forceinline__ double rcp_newton(double x) {
  const double sc = pow2_inverse(x);
  const double x1 = x * sc;                                  // in [1, 2)
  double y = (double)(1.0f / (float)x1);
  y = y * fma(-x1, y, 2.0);
  y = y * fma(-x1, y, 2.0);
  return y * sc;
}

// Forms the Householder reflector of column c (held by this warp: value a[u] at row lane + 32 u,
// m rows) that zeroes the rows below c, and publishes v = (0, .., 0, 1, x / (alpha - beta)) into
// v_out[0, vlen), tau = (beta - alpha) / beta and the diagonal entry beta of R.  With
// beta = -sign(alpha) ||a||, tau = 1 + |alpha| / ||a|| and 1 / (alpha - beta) =
// sign(alpha) / (|alpha| + ||a||), so one reciprocal square root and one reciprocal (rsqrt_newton,
// rcp_newton) form the reflector.  A column whose rows below c are already zero gets tau = 0 and
// keeps its diagonal entry.  Returns false when the column norm is not finite.
template <int kRpl>
__device__ __forceinline__ bool reflector_publish_d(const double (&a)[kRpl], int c, int m, double* v_out, int vlen,
                                                    double* tau_out, double* rdiag) {
  const int lane = threadIdx.x & 31;
  double t0 = 0.0, t1 = 0.0, alpha = 0.0;
#pragma unroll
  for (int u = 0; u < kRpl; ++u) {
    const int i = lane + 32 * u;
    if (i > c && i < m) {
      if (u & 1) t1 = fma(a[u], a[u], t1);
      else t0 = fma(a[u], a[u], t0);
    }
    if (i == c) alpha = a[u];
  }
  const double t2 = warp_sum_d(t0 + t1);
  alpha = __shfl_sync(0xffffffffu, alpha, c & 31);
  const double z = fma(alpha, alpha, t2);
  const bool finite = isfinite(z);
  const bool reflect = t2 > 0.0 && finite && pow2_inverse(z) > 0.0;
  double tau = 0.0, sc = 0.0, beta = alpha;
  if (reflect) {
    const double inv_n = rsqrt_newton(z);
    const double nrm = z * inv_n;
    const double aa = fabs(alpha);
    tau = fma(aa, inv_n, 1.0);
    const double r = rcp_newton(aa + nrm);
    sc = alpha >= 0.0 ? r : -r;
    beta = alpha >= 0.0 ? -nrm : nrm;
  }
#pragma unroll
  for (int u = 0; u < kRpl; ++u) {
    const int i = lane + 32 * u;
    if (i < vlen) v_out[i] = i < c ? 0.0 : (i == c ? 1.0 : (i < m ? sc * a[u] : 0.0));
  }
  if (lane == 0) {
    *tau_out = tau;
    rdiag[c] = beta;
  }
  return finite;
}

// ----------------------------------------------------------------------------- TSQR block (float64)
// Householder QR of a rows x cols block of a float64 source read through a two-level row index
// (rows <= 32 kRpl, cols <= kWarps kSlots); only the triangular factor is kept.  The block is staged
// through shared memory (coalesced along whichever index is contiguous in the source) and then
// lives in registers: column l in warp l % kWarps (slot l / kWarps), lane L holds rows L + 32 u.  Each step j
// reads the published reflector v_j and tau_j, every warp updates its columns l > j, and the warp
// owning column j + 1 forms and publishes the next reflector: one barrier per column.
constexpr int kT64LoadBatch = 8;

template <int kRpl, int kSlots, int kWarps>
__global__ void __launch_bounds__(32 * kWarps, 1) tsqr_f64_kernel(const TsqrJob* __restrict__ jobs, Bases bases) {
  constexpr int kThreads = 32 * kWarps;
  constexpr int kBlockRows = 32 * kRpl;
  extern __shared__ double smem_t64[];
  __shared__ double vbuf[2][kBlockRows];
  __shared__ double sh_tau[2];
  __shared__ double rdiag[kWarps * kSlots];
  __shared__ int64_t rowoff[kBlockRows];
  const TsqrJob& J = jobs[blockIdx.x];
  // a gated block (the Householder fallback of CholeskyQR3) runs only when its job asked for it
  if (J.gate.base != B_NONE && *at<const int32_t>(bases, J.gate) == 0) return;
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
  for (int e0 = 0; e0 < mb; e0 += kT64LoadBatch * kThreads) {
    double v[kT64LoadBatch];
    int dst[kT64LoadBatch];
#pragma unroll
    for (int u = 0; u < kT64LoadBatch; ++u) {
      const int e = e0 + u * kThreads + threadIdx.x;
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
    const int l = warp + kWarps * sl;
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
    // row slots that can hold a nonzero of v_j: rows below the block's end, at or below row j, and
    // for a stack of tri interleaved triangular factors (row i = factor + tri r) with r <= j
    unsigned umask = 0;
#pragma unroll
    for (int u = 0; u < kRpl; ++u)
      if (32 * u < m && 32 * u + 31 >= j && (J.tri == 0 || 32 * u < J.tri * (j + 1))) umask |= 1u << u;
    apply_reflector_d<kRpl, kSlots, kWarps>(a, vj, tau, j, b, umask);
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
      const int l = warp + kWarps * sl;
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
    const int c = warp + kWarps * sl;
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
// One-sided (Hestenes) Jacobi with the round-robin ordering: each round rotates b/2 disjoint column
// pairs (kJ64Lanes lanes per pair) until they are orthogonal.  It runs on the columns of X = R^T for
// the b x b factor R of H_(n)^T: at convergence X J = U Sigma, and U (the normalized columns) holds the
// right singular vectors of R, i.e. the left singular vectors of H_(n).  Then the singular values
// (column norms) are sorted, the rank rule of Alg. 2 applied and P = the leading columns of U,
// sign-fixed (largest-magnitude entry positive), zero-padded to rmax.

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

// Column pair of group k in round `round` of the circle ordering over m (even) columns: pair 0 is
// (round, m - 1), pair k > 0 is ((round + k) mod (m - 1), (round - k) mod (m - 1)); p < q.
__device__ __forceinline__ void jacobi_pair(int k, int round, int m, int& p, int& q) {
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
}

// tan(theta) of the Jacobi rotation, t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) with zeta = num / den
// (den != 0), evaluated in float32 after scaling num and den by the same power of two.  The angle only
// steers convergence (a t off by float32 rounding leaves a float32-relative residual coupling that the
// next sweep removes); the rotation built from t is exactly orthogonal in float64 in any case.  When a
// rotation is taken, |zeta| < 1 / (16 eps thr), so the scaled values stay in float32 range.
__device__ __forceinline__ double jacobi_tangent(double num, double den) {
  const double sc = pow2_inverse(fabs(den));
  float z;
  if (sc > 0.0) {
    z = (float)(num * sc) / (float)(den * sc);
  } else {
    z = (float)(num / den);
  }
  const float az = fabsf(z);
  const float tm = az > 1e18f ? 0.5f / az : 1.f / (az + sqrtf(fmaf(az, az, 1.f)));
  return (double)copysignf(tm, z);
}

// Float64 sweeps on the columns of A (ld doubles apart, 16-byte aligned) until no pair rotates or
// max_sweeps; returns the sweeps run.  Rotates while |a_p . a_q| > b eps ||a_p|| ||a_q||, skipping
// columns at the float64 noise floor (norm <= 8 eps max norm): their couplings are rounding noise.
// The rotation angle is that of the symmetric 2 x 2 Schur decomposition of the pair's Gram block
// (Golub & Van Loan), t = tan(theta) from zeta = (beta - alpha) / (2 gamma).
//
// Each column is kept as d_c a_c (a scale and a stored vector) with its squared norm n_c tracked
// through the rotations: the rotation P' = c (P - t Q), Q' = c (Q + t P) becomes
//   a_p <- a_p - (t d_q / d_p) a_q,  a_q <- a_q + (t d_p / d_q) a_p,  d_p, d_q <- c d_p, c d_q,
//   n_p <- n_p - t gamma,  n_q <- n_q + t gamma,
// so a pair costs one dot product (gamma) and one FMA per stored element, instead of three dot
// products and two multiplies plus two FMAs (on GB300 the FP64 pipe, at 1/64 of the float32 rate,
// is the bound).  At the start of every sweep the scales are folded into the vectors and the norms
// recomputed, which bounds the drift of both.  The rotation is computed by the first lane of each
// group and broadcast, with the tangent in float32 (jacobi_tangent) and c = 1 / sqrt(1 + t^2)
// refined to float64 by two Newton steps, so the chain of dependent float64 operations that bounds
// a round's latency is a small fraction of a float64 division-and-square-root evaluation.  A pair is
// visited once per sweep; when neither of its columns has rotated since its previous visit (in the
// previous sweep or earlier in this one) it is still orthogonal and is skipped without loading it.
// dsc, dinv and nsq hold m doubles each, flags 2 m ints.
// kChunks: 2-row chunks per lane (8 lanes per pair), enough for b rows; a smaller count than the
// largest basis keeps the float64 pipe off padding rows (b <= 64 needs 4 of 6).
template <int kChunks>
__device__ int jacobi_sweeps_f64(double* A, int ld, int b, int m, int max_sweeps, double noise2, int* sh_rot,
                                 double* dsc, double* dinv, double* nsq, int* flags) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int sub = lane % kJ64Lanes;
  const int lead = lane - sub;
  const int k = threadIdx.x / kJ64Lanes;
  const int pairs = m / 2;
  const double thr = (double)b * 1.1102230246251565e-16, thr2 = thr * thr;
  __shared__ double sh_g[TKS_MAX_BASIS / 2], sh_mp[TKS_MAX_BASIS / 2], sh_mq[TKS_MAX_BASIS / 2];
  __shared__ int sh_act[TKS_MAX_BASIS / 2];
  int* rot_prev = flags;       // column rotated during the previous sweep (all set before the first)
  int* rot_cur = flags + m;    // column rotated so far in this sweep
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    rot_prev[c] = 1;
    rot_cur[c] = 0;
    dsc[c] = 1.0;
    dinv[c] = 1.0;
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    // fold the scales into the vectors and recompute the squared norms
    for (int c = warp; c < b; c += nw) {
      const double dc = dsc[c];
      double s2 = 0.0;
      for (int i = lane; i < b; i += 32) {
        const double v = dc * A[i + c * ld];
        A[i + c * ld] = v;
        s2 = fma(v, v, s2);
      }
      s2 = warp_sum_d(s2);
      if (lane == 0) {
        nsq[c] = s2;
        dsc[c] = 1.0;
        dinv[c] = 1.0;
      }
    }
    if (threadIdx.x == 0) *sh_rot = 0;
    __syncthreads();
    int any = 0;
    for (int round = 0; round < m - 1; ++round) {
      int p, q;
      jacobi_pair(k, round, m, p, q);
      bool valid = k < pairs && q < b;
      if (valid) valid = (rot_prev[p] | rot_prev[q] | rot_cur[p] | rot_cur[q]) != 0;
      if (!valid) p = q = 0;
      double* ap = A + p * ld;
      double* aq = A + q * ld;
      double2 x[kChunks], y[kChunks];
      double g = 0.0;
      if (__any_sync(0xffffffffu, valid)) {
        double g0 = 0.0, g1 = 0.0;
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
          const int i = 2 * (sub + kJ64Lanes * u);
          const bool in = valid && i < b;
          x[u] = in ? *reinterpret_cast<const double2*>(ap + i) : make_double2(0.0, 0.0);
          y[u] = in ? *reinterpret_cast<const double2*>(aq + i) : make_double2(0.0, 0.0);
          g0 = fma(x[u].x, y[u].x, g0);
          g1 = fma(x[u].y, y[u].y, g1);
        }
        g = g0 + g1;
#pragma unroll
        for (int o = kJ64Lanes / 2; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o, kJ64Lanes);
      }
      if (sub == 0 && k < pairs) {
        sh_g[k] = g;
        sh_act[k] = valid ? 1 : 0;
      }
      __syncthreads();
      // one warp forms every pair's rotation, lane = pair: the scalar float64 work of a round then
      // issues as full warps instead of one lane in eight (the float64 pipe counts issued warps)
      if (warp == 0) {
        for (int pk = lane; pk < pairs; pk += 32) {
          if (!sh_act[pk]) continue;
          int pp, qq;
          jacobi_pair(pk, round, m, pp, qq);
          int act = 0;
          const double dp = dsc[pp], dq = dsc[qq];
          const double al = nsq[pp], be = nsq[qq];
          const double ga = dp * dq * sh_g[pk];
          // |gamma| > thr sqrt(alpha beta), evaluated on values scaled by a power of two near
          // 1 / max(alpha, beta) so that neither product under- or overflows
          const double sc = pow2_inverse(fmax(al, be));
          const double a1 = al * sc, b1 = be * sc, g1 = ga * sc;
          if (sc > 0.0 && g1 * g1 > thr2 * a1 * b1 && fmin(al, be) > noise2) {
            const double t = jacobi_tangent(be - al, 2.0 * ga);
            // c = 1 / sqrt(w), w = 1 + t^2, from the float32 estimate and two Newton steps (float64
            // accuracy: c^2 (1 + t^2) = 1 is what makes the rotation orthogonal)
            const double w = fma(t, t, 1.0), hw = 0.5 * w;
            double c = (double)rsqrtf((float)w);
            c = c * fma(-hw * c, c, 1.5);
            c = c * fma(-hw * c, c, 1.5);
            const double c2 = c * c, wc = w * c;   // c^2 and sqrt(w)
            const double ip = dinv[pp], iq = dinv[qq];
            sh_mp[pk] = t * dq * ip;
            sh_mq[pk] = t * dp * iq;
            dsc[pp] = c * dp;
            dsc[qq] = c * dq;
            dinv[pp] = ip * wc;
            dinv[qq] = iq * wc;
            // the new squared norms for this t (exactly the rotated columns' norms, whatever t is)
            nsq[pp] = c2 * fma(t, fma(t, be, -2.0 * ga), al);
            nsq[qq] = c2 * fma(t, fma(t, al, 2.0 * ga), be);
            rot_cur[pp] = rot_cur[qq] = 1;
            act = 1;
          }
          sh_act[pk] = act;
        }
      }
      __syncthreads();
      const int act = (k < pairs) ? sh_act[k] : 0;
      if (act) {
        const double mp = sh_mp[k], mq = sh_mq[k];
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
          const int i = 2 * (sub + kJ64Lanes * u);
          if (i < b) {
            const double2 a0 = x[u], b0 = y[u];
            *reinterpret_cast<double2*>(ap + i) = make_double2(fma(-mp, b0.x, a0.x), fma(-mp, b0.y, a0.y));
            *reinterpret_cast<double2*>(aq + i) = make_double2(fma(mq, a0.x, b0.x), fma(mq, a0.y, b0.y));
          }
        }
        any = 1;
      }
      __syncthreads();
    }
    if (any) *sh_rot = 1;
    __syncthreads();
    const int rot = *sh_rot;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      rot_prev[c] = rot_cur[c];
      rot_cur[c] = 0;
    }
    __syncthreads();
    if (!rot) break;
  }
  // fold the last scales in: A holds the rotated columns
  for (int c = warp; c < b; c += nw) {
    const double dc = dsc[c];
    for (int i = lane; i < b; i += 32) A[i + c * ld] *= dc;
  }
  __syncthreads();
  return sweep;
}

// Largest squared column norm of the b x b matrix A (columns ld apart) over the CTA, as a double.
__device__ double max_col_norm2(const double* A, int ld, int b, double* slot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) *slot = 0.0;
  __syncthreads();
  for (int c = warp; c < b; c += nw) {
    double s2 = 0.0;
    for (int i = lane; i < b; i += 32) s2 = fma(A[i + c * ld], A[i + c * ld], s2);
    s2 = warp_sum_d(s2);
    // non-negative doubles order like their bit patterns (a NaN sorts above them and stays)
    if (lane == 0) atomicMax(reinterpret_cast<unsigned long long*>(slot), (unsigned long long)__double_as_longlong(s2));
  }
  __syncthreads();
  const double v = *slot;
  __syncthreads();
  return v;
}

// The one-sided Jacobi runs on X = R^T: its left singular vectors are the right singular vectors of R,
// i.e. the left singular vectors of H_(n), and at convergence they are the normalized columns of the
// rotated X, so no rotation needs to be accumulated in float64.  (On a triangular factor from QR, the
// sweeps on R^T also converge in about half the sweeps that R itself needs.)  Kept columns whose norm
// is at the float64 noise floor carry no direction; they are replaced by an orthonormal completion.
template <int kChunks>
__global__ void __launch_bounds__(kJ64Threads, 1) svd_jacobi_f64_kernel(const SvdJob* __restrict__ jobs, Bases bases,
                                                                   Status* status) {
  extern __shared__ double sm64[];
  const SvdJob& J = jobs[blockIdx.x];
  const int b = J.b;
  const int m = b + (b & 1);
  const int ld = m;                 // even: columns start 16-byte aligned; rows in [b, ld) stay zero
  double* A = sm64;                 // m x ld: X = R^T, rotated
  double* nrm = A + m * ld;
  double* dsc = nrm + m;            // column scales of the float64 sweeps
  double* dinv = dsc + m;           // their inverses
  double* nsq = dinv + m;           // tracked squared column norms
  int* order = reinterpret_cast<int*>(nsq + m);
  int* flags = order + m;           // 2 m
  __shared__ int sh_rot, sh_rank, sh_fill;
  __shared__ double red[32];
  __shared__ double sh_max;
  const double eps = 1.1102230246251565e-16;
  const double* Rg = at<double>(bases, J.R);   // X[i, k] = R[k, i] = Rg[k + b i]
  for (int e = threadIdx.x; e < m * ld; e += blockDim.x) {
    const int r = e % ld, c = e / ld;
    A[e] = (r < b && c < b) ? Rg[c + r * b] : 0.0;
  }
  __syncthreads();
  const double noise2 = max_col_norm2(A, ld, b, &sh_max) * (8.0 * eps) * (8.0 * eps);
  const int sweep = jacobi_sweeps_f64<kChunks>(A, ld, b, m, kJ64Sweeps, noise2, &sh_rot, dsc, dinv, nsq, flags);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
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
  for (int i = threadIdx.x; i < b; i += blockDim.x) {
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
    if (J.err.base != B_NONE) {
      // the energy this mode's truncation discards; with the first mode's total, the ST-HOSVD's
      // relative error (the discarded parts of successive modes are orthogonal)
      double* er = at<double>(bases, J.err);
      double dis = 0.0;
      for (int i = r; i < b; ++i) dis += (double)nrm[order[i]];
      if (J.first_mode) er[0] = (double)tot;
      er[1 + J.mode] = dis;
    }
    // kept columns from the first one at the noise floor on carry no direction
    int fill = r;
    for (int t = 0; t < r; ++t)
      if (!(nrm[order[t]] > noise2)) {
        fill = t;
        break;
      }
    sh_fill = fill;
    *at<int32_t>(bases, J.rank) = r;
    if (!isfinite(tot)) record_status_64(status, TKS_ENONFINITE);
    if (sweep >= kJ64Sweeps) record_status_64(status, TKS_ENOCONV);
  }
  __syncthreads();
  const int r = sh_rank, fill = sh_fill;
  double* P = at<double>(bases, J.P);
  // P[:, t] = the normalized column of rank t, sign-fixed (largest-magnitude entry positive)
  for (int t = warp; t < J.rmax; t += nw) {
    if (t >= fill) {
      for (int i = lane; i < b; i += 32) P[i + (int64_t)t * b] = 0.0;
      continue;
    }
    const int src = order[t];
    const double inv = 1.0 / sqrt(nrm[src]);
    double best = 0.0;
    for (int i = lane; i < b; i += 32) {
      const double v = A[i + src * ld];
      if (fabs(v) > fabs(best)) best = v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double other = __shfl_xor_sync(0xffffffffu, best, o);
      if (fabs(other) > fabs(best) || (fabs(other) == fabs(best) && other > best)) best = other;
    }
    const double sc = (best < 0.0) ? -inv : inv;
    for (int i = lane; i < b; i += 32) P[i + (int64_t)t * b] = sc * A[i + src * ld];
  }
  if (fill >= r) return;
  __syncthreads();
  // orthonormal completion of columns [fill, r) (one warp; only rank-deficient H reaches this): for
  // each, the unit vector e_j with the largest part orthogonal to the columns before it,
  // 1 - sum_u P[j, u]^2 >= (b - t) / b, orthogonalized by two Gram-Schmidt passes and normalized
  if (warp == 0) {
    for (int t = fill; t < r; ++t) {
      double* pt = P + (int64_t)t * b;
      double best = -1.0;
      int jbest = 0;
      for (int j = lane; j < b; j += 32) {
        double s2 = 0.0;
        for (int u = 0; u < t; ++u) s2 = fma(P[j + (int64_t)u * b], P[j + (int64_t)u * b], s2);
        if (1.0 - s2 > best) { best = 1.0 - s2; jbest = j; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, jbest, o);
        if (ob > best || (ob == best && oj < jbest)) { best = ob; jbest = oj; }
      }
      for (int i = lane; i < b; i += 32) pt[i] = (i == jbest) ? 1.0 : 0.0;
      __syncwarp();
      for (int pass = 0; pass < 2; ++pass) {
        for (int u = 0; u < t; ++u) {
          const double* pu = P + (int64_t)u * b;
          double d = 0.0;
          for (int i = lane; i < b; i += 32) d = fma(pu[i], pt[i], d);
          d = warp_sum_d(d);
          for (int i = lane; i < b; i += 32) pt[i] = fma(-d, pu[i], pt[i]);
          __syncwarp();
        }
      }
      double n2 = 0.0;
      for (int i = lane; i < b; i += 32) n2 = fma(pt[i], pt[i], n2);
      n2 = warp_sum_d(n2);
      const double inv = 1.0 / sqrt(n2);
      for (int i = lane; i < b; i += 32) pt[i] *= inv;
      __syncwarp();
    }
  }
}

size_t svd64_smem(int bmax) {
  const int m = bmax + (bmax & 1);
  return (size_t)m * m * sizeof(double) + (size_t)4 * m * sizeof(double) + (size_t)3 * m * sizeof(int);
}

size_t tsqr64_smem(int rows, int cols) { return (size_t)(rows + 1) * cols * sizeof(double); }

// ----------------------------------------------------------------------------- mode products (float64)
// Y[l + L (c + rmax r)] = sum_a X[l + L (a + b r)] P[a + b c] for l < L, r < Rr, c < rmax: the
// ST-HOSVD truncation H <- H x_n P_n^T (X = H, fibres q = (l, r)) and the factors U~_n = Q_n P_n
// (X = Q_n, L = n_n, Rr = 1).  A GEMM whose rows are the fibres, with K = b and N = rmax small: a
// CTA takes kTtmF fibres and every column, stages the fibre tile (b x kTtmF) and P in shared memory
// (coalesced along a when L = 1, along l otherwise), and each thread accumulates 4 fibres x
// ceil(rmax / 16) columns over a in order.  Columns are tiled by 16, so at rmax = 48 no product is
// wasted on padding (a general 64 x 64 tile computes 64 columns for 48); the FP64 pipe is the bound.
constexpr int kTtmF = 64;                   // fibres per CTA
constexpr int kTtmThreads = 256;            // 16 fibre lanes x 16 column lanes
constexpr int kTtmXs = kTtmF + 1;           // padded row of the fibre tile

// kCj = column groups of 16 (columns of the launch's widest job, rounded up); b is padded to a
// multiple of 4 with zero rows so the reduction loop unrolls by four.
template <int kCj>
__global__ void __launch_bounds__(kTtmThreads) ttm_f64_kernel(const TtmJob* __restrict__ jobs, int njobs,
                                                             Bases bases) {
  constexpr int kCols = 16 * kCj;
  extern __shared__ double tsm64[];
  __shared__ int64_t fib_off[kTtmF];
  const int lo = tile_job(jobs, njobs, (int)blockIdx.x);
  const TtmJob& J = jobs[lo];
  const int b = J.b, rmax = J.rmax;
  const int bp = (b + 3) & ~3;
  const int64_t L = J.L, nfib = J.L * J.Rr;
  const int64_t q0 = (int64_t)(blockIdx.x - J.tile_begin) * kTtmF;
  const int nq = (int)(nfib - q0 < kTtmF ? nfib - q0 : kTtmF);
  double* Ps = tsm64;                     // [a][c], zero for c >= rmax and a >= b
  double* Xs = Ps + (size_t)bp * kCols;   // [a][q], row kTtmXs, zero for a >= b and q >= nq
  const double* X = at<double>(bases, J.X);
  const double* P = at<double>(bases, J.P);
  double* Y = at<double>(bases, J.Y);
  for (int e = threadIdx.x; e < bp * kCols; e += kTtmThreads) {
    const int a = e % bp, c = e / bp;
    Ps[a * kCols + c] = (c < rmax && a < b) ? P[a + (int64_t)b * c] : 0.0;
  }
  if (L == 1) {
    // fibres are contiguous runs of b elements starting at (q0 + q) b
    for (int e = threadIdx.x; e < bp * kTtmF; e += kTtmThreads) {
      const int q = e / bp, a = e - q * bp;
      Xs[a * kTtmXs + q] = (q < nq && a < b) ? X[(q0 + q) * b + a] : 0.0;
    }
  } else {
    for (int q = threadIdx.x; q < kTtmF; q += kTtmThreads) {
      const int64_t f = q0 + q, r = f / L, l = f - r * L;
      fib_off[q] = l + L * (int64_t)b * r;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < bp * kTtmF; e += kTtmThreads) {
      const int q = e % kTtmF, a = e / kTtmF;
      Xs[a * kTtmXs + q] = (q < nq && a < b) ? X[fib_off[q] + L * a] : 0.0;
    }
  }
  __syncthreads();
  const int tq = threadIdx.x % 16, tc = threadIdx.x / 16;
  double acc[4][kCj];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < kCj; ++j) acc[i][j] = 0.0;
  for (int a0 = 0; a0 < bp; a0 += 4) {
#pragma unroll
    for (int da = 0; da < 4; ++da) {
      const int a = a0 + da;
      double xv[4], pv[kCj];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = Xs[a * kTtmXs + tq + 16 * i];
#pragma unroll
      for (int j = 0; j < kCj; ++j) pv[j] = Ps[a * kCols + tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < kCj; ++j) acc[i][j] = fma(xv[i], pv[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int q = tq + 16 * i;
    if (q >= nq) continue;
    const int64_t f = q0 + q, r = f / L, l = f - r * L;
    double* y = Y + l + L * (int64_t)rmax * r;
#pragma unroll
    for (int j = 0; j < kCj; ++j) {
      const int c = tc + 16 * j;
      if (c < rmax) y[L * c] = acc[i][j];
    }
  }
}

size_t ttm64_smem(int bmax) {
  const int bp = (bmax + 3) & ~3, cols = 16 * ((bmax + 15) / 16);
  return (size_t)bp * cols * sizeof(double) + (size_t)bp * kTtmXs * sizeof(double);
}

// ----------------------------------------------------------------------------- CholeskyQR3 steps
// One pass of shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto and Yanagisawa 2020) for
// the triangular factor of X = H_(n)^T (P x b, b <= 64), one CTA per job, in float64:
//   pass 1: R1 = chol(G + s I), s = 11 (P b + b (b + 1)) u ||X||_F^2 (||X||_F^2 = trace G): the shift
//           keeps the factorization defined for any conditioning and leaves X R1^-1 with a condition
//           number near u^-1/2;
//   pass 2, 3: R = chol(G) of the re-formed X R^-1 (CholeskyQR2), which restores orthogonality to
//           rounding;  R = R3 R2 R1 is then a backward-stable triangular factor of X.
// Every pass writes Rinv = R^-1 (upper, column-major) for the next X <- X Rinv and accumulates
// Racc <- R Racc; the last writes Racc to Rout.  A pivot that is not positive (pass 1) or below 1e-12
// of its diagonal entry (passes 2, 3: X R^-1 is too ill-conditioned for CholeskyQR2, e.g. a rank-
// deficient unfolding) sets *fallback, and the Householder TSQR factors X instead; later passes of a
// failed job only write an identity Rinv.
//
// Layout: thread (r, ty) = (threadIdx % 64, threadIdx / 64) owns row r of every triangle and the
// columns c = ty (mod 4), so a warp reads one column of the pivot row (a broadcast) and 32 consecutive
// rows of the matrix it updates (no bank conflicts), and every elimination step costs one barrier.
// The factor is kept as G = U^T D^-1 U with U's rows unscaled (d_j = U[j][j], the pivots), so a step
// needs no square root:  R = D^-1/2 U,  R^-1 = Z D^-1/2 with Z the inverse of the unit triangle D^-1 U.
constexpr int kCholThreads = 256;
constexpr int kCholTri = 64 * 65 / 2;   // entries of a 64 x 64 upper triangle
constexpr size_t kCholSmem = (3 * 64 * 65 + 2 * 64) * sizeof(double);

// Upper-triangle index tables (r | c << 8): by row, rows from the last up (the trailing triangle
// of elimination step j is the prefix of (b - 1 - j)(b - j) / 2 entries), and by diagonal c - r
// (entries of one diagonal have dot products of equal length).  The float64 pipe issues per warp,
// so the loops run over these flat lists with every lane busy rather than over predicated rows.
__device__ __forceinline__ void chol_tables(int b, uint16_t* tri_r, uint16_t* tri_d) {
  const int t = threadIdx.x;
  if (t < b) {
    const int w = b - 1 - t;                       // rows after t
    const int off_r = w * (w + 1) / 2;
    for (int c = t; c < b; ++c) tri_r[off_r + (c - t)] = (uint16_t)(t | (c << 8));
    const int d = t, off_d = d * b - d * (d - 1) / 2;
    for (int r = 0; r + d < b; ++r) tri_d[off_d + r] = (uint16_t)(r | ((r + d) << 8));
  }
}

__global__ void __launch_bounds__(kCholThreads, 1) chol_step_kernel(const CholJob* __restrict__ jobs, Bases bases,
                                                                Status* status) {
  extern __shared__ double cs64[];
  const CholJob& J = jobs[blockIdx.x];
  const int b = J.b, ld = b + 1;
  double* A = cs64;                 // G, then U (upper triangle), then R (zero below the diagonal)
  double* Z = A + b * ld;           // (D^-1 U)^-1, unit upper triangular
  double* Ra = Z + b * ld;          // Racc of the previous passes
  double* dv = Ra + b * ld;         // pivots d_j
  double* dg = dv + 64;             // the diagonal of G
  __shared__ double rdv[64];        // 1 / d_j
  __shared__ double fr[64];         // the multipliers of one step
  __shared__ uint16_t tri_r[kCholTri], tri_d[kCholTri];
  __shared__ int sh_fail;
  const int tid = threadIdx.x;
  int32_t* fb = at<int32_t>(bases, J.fallback);
  double* Rinv = at<double>(bases, J.Rinv);
  double* Racc = at<double>(bases, J.Racc);
  const double* G = at<const double>(bases, J.G);
  if (tid == 0) sh_fail = J.pass == 1 ? 0 : *fb;
  for (int e = tid; e < b * b; e += kCholThreads) {
    const int i = e % b, c = e / b;
    A[i + ld * c] = G[e];
    Z[i + ld * c] = i == c ? 1.0 : 0.0;
    if (J.pass > 1) Ra[i + ld * c] = Racc[e];
    if (i == c) dg[i] = G[e];
  }
  chol_tables(b, tri_r, tri_d);
  __syncthreads();
  bool fail = sh_fail != 0;         // the same value in every thread from here on
  if (!fail && J.shift) {
    double tr = 0.0;
    for (int i = 0; i < b; ++i) tr += dg[i];
    const double shift = 11.0 * ((double)J.P * b + (double)b * (b + 1)) * 1.1102230246251565e-16 * tr;
    fail = !isfinite(tr);
    if (!fail && tid < b) A[tid + ld * tid] += shift;
    __syncthreads();
  }
  // right-looking elimination: step j takes the pivot d = U[j][j] and updates the trailing triangle,
  // A[r][c] -= (A[j][r] / d) A[j][c] for j < r <= c; every thread reads the same pivot, so all leave
  // together.  Each step's one division is taken by the thread that finishes the next pivot.
  if (!fail && tid == 0) rdv[0] = 1.0 / A[0];
  if (!fail) __syncthreads();
  for (int j = 0; j < b && !fail; ++j) {
    const double d = A[j + ld * j];
    const double bound = J.pivot_tol * dg[j];
    if (!(d > bound) || !isfinite(d)) {
      fail = true;
      break;
    }
    if (tid == 0) dv[j] = d;
    if (tid > j && tid < b) fr[tid] = A[j + ld * tid] * rdv[j];
    __syncthreads();
    const int w = b - 1 - j, n = w * (w + 1) / 2;
    for (int e = tid; e < n; e += kCholThreads) {
      const int r = tri_r[e] & 255, c = tri_r[e] >> 8;
      const double v = fma(-fr[r], A[j + ld * c], A[r + ld * c]);
      A[r + ld * c] = v;
      if (c == r && r == j + 1) rdv[r] = 1.0 / v;
    }
    __syncthreads();
  }
  if (fail) {
    // this job takes the Householder fallback: an identity Rinv keeps the following products harmless
    for (int e = tid; e < b * b; e += kCholThreads) Rinv[e] = (e % b == e / b) ? 1.0 : 0.0;
    if (tid == 0) *fb = 1;
    return;
  }
  // Z from the bottom: step k subtracts (U[i][k] / d_i) Z[k][:] from the rows i < k (row k is final);
  // the k x (b - k) block is one flat list, e -> (e mod k, k + e div k) with the quotient from a float32
  // reciprocal (exact here: e < 4096 and k <= 64 keep the product 2^-22 away from the next integer)
  for (int k = b - 1; k > 0; --k) {
    if (tid < k) fr[tid] = A[tid + ld * k] * rdv[tid];
    __syncthreads();
    const float rk = 1.0f / (float)k;
    const int n = k * (b - k);
    for (int e = tid; e < n; e += kCholThreads) {
      const int qd = (int)(((float)e + 0.5f) * rk), i = e - qd * k, c = k + qd;
      Z[i + ld * c] = fma(-fr[i], Z[k + ld * c], Z[i + ld * c]);
    }
    __syncthreads();
  }
  // R = D^-1/2 U in place, Rinv = Z D^-1/2 (row a times 2^xexp[a] when X's digits carry column exponents)
  __shared__ int xe[64];
  if (tid < b) {
    dg[tid] = sqrt(rdv[tid]);
    xe[tid] = J.xexp.base != B_NONE ? at<const int32_t>(bases, J.xexp)[tid] : 0;
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += kCholThreads) {
    const int i = e % b, c = e / b;
    A[i + ld * c] = i <= c ? A[i + ld * c] * dg[i] : 0.0;
    Rinv[e] = i <= c ? scalbn(Z[i + ld * c] * dg[c], xe[i]) : 0.0;
  }
  __syncthreads();
  // Racc <- R Racc (pass 1: Racc = R); the last pass writes it to Rout when one is given.  Both are
  // upper triangular, so T[r][c] = sum_{k = r..c} R[r][k] Racc[k][c], taken diagonal by diagonal.
  double* out = (J.last && J.Rout.base != B_NONE) ? at<double>(bases, J.Rout) : Racc;
  if (J.pass == 1) {
    for (int e = tid; e < b * b; e += kCholThreads) out[e] = A[(e % b) + ld * (e / b)];
  } else {
    const int n = b * (b + 1) / 2;
    for (int e = tid; e < n; e += kCholThreads) {
      const int r = tri_d[e] & 255, c = tri_d[e] >> 8;
      double acc = 0.0;
      for (int k = r; k <= c; ++k) acc = fma(A[r + ld * k], Ra[k + ld * c], acc);
      out[r + b * c] = acc;
    }
    for (int e = tid; e < b * b; e += kCholThreads)
      if (e % b > e / b) out[e] = 0.0;
  }
  if (J.pass == 1 && tid == 0) *fb = 0;
  (void)status;
}

}  // namespace

namespace {
__global__ void trunc_err_kernel(const TruncErrJob* __restrict__ jobs, int njobs, Bases bases) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= njobs) return;
  const TruncErrJob& J = jobs[j];
  const double* er = at<const double>(bases, J.err);
  double dis = 0.0;
  for (int n = 0; n < J.d; ++n) dis += er[1 + n];
  *at<double>(bases, J.out) = er[0] > 0.0 ? sqrt(dis / er[0]) : 0.0;
}
}  // namespace

void launch_trunc_err(const TruncErrJob* jobs, int njobs, const Bases& bases, cudaStream_t stream) {
  trunc_err_kernel<<<(njobs + 127) / 128, 128, 0, stream>>>(jobs, njobs, bases);
}

// At least twice the columns, so that every TSQR level shrinks the stack of factors.
int tsqr64_block_rows(int max_cols) { return max_cols <= 64 ? 256 : 192; }

cudaError_t prepare_la64(int bmax) {
  cudaError_t e0 = cudaFuncSetAttribute(chol_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kCholSmem);
  if (e0 != cudaSuccess) return e0;
  cudaError_t e = cudaFuncSetAttribute(svd_jacobi_f64_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)svd64_smem(bmax));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(svd_jacobi_f64_kernel<kJ64Chunks>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)svd64_smem(bmax));
  if (e != cudaSuccess) return e;
  const void* ttm_kernels[] = {reinterpret_cast<const void*>(ttm_f64_kernel<1>),
                               reinterpret_cast<const void*>(ttm_f64_kernel<2>),
                               reinterpret_cast<const void*>(ttm_f64_kernel<3>),
                               reinterpret_cast<const void*>(ttm_f64_kernel<4>),
                               reinterpret_cast<const void*>(ttm_f64_kernel<5>),
                               reinterpret_cast<const void*>(ttm_f64_kernel<6>)};
  for (const void* k : ttm_kernels) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ttm64_smem(bmax));
    if (e != cudaSuccess) return e;
  }
  const void* kernels[] = {reinterpret_cast<const void*>(tsqr_f64_kernel<8, 2, 16>),
                           reinterpret_cast<const void*>(tsqr_f64_kernel<8, 3, 16>),
                           reinterpret_cast<const void*>(tsqr_f64_kernel<8, 4, 16>),
                           reinterpret_cast<const void*>(tsqr_f64_kernel<6, 6, 16>)};
  // the largest staging tile of any instantiation: 256 x 64 or 192 x 96
  const size_t tile = std::max(tsqr64_smem(256, 64), tsqr64_smem(192, 96));
  for (const void* k : kernels) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void launch_tsqr_f64(const TsqrJob* jobs, int njobs, int max_cols, const Bases& bases, cudaStream_t stream) {
  // the smallest instantiation that covers max_cols: 16 warps hold up to 64 columns of a 256-row
  // block (32 doubles per thread), 96 columns of a 192-row block (36); 768-thread variants with fewer
  // columns per warp were measured slower (more instructions per column step)
  if (max_cols <= 32) {
    tsqr_f64_kernel<8, 2, 16><<<njobs, 512, tsqr64_smem(256, 32), stream>>>(jobs, bases);
  } else if (max_cols <= 48) {
    tsqr_f64_kernel<8, 3, 16><<<njobs, 512, tsqr64_smem(256, 48), stream>>>(jobs, bases);
  } else if (max_cols <= 64) {
    tsqr_f64_kernel<8, 4, 16><<<njobs, 512, tsqr64_smem(256, 64), stream>>>(jobs, bases);
  } else {
    tsqr_f64_kernel<6, 6, 16><<<njobs, 512, tsqr64_smem(192, 96), stream>>>(jobs, bases);
  }
}

void launch_svd_f64(const SvdJob* jobs, int njobs, int bmax, const Bases& bases, Status* status,
                    cudaStream_t stream) {
  const int pairs = (bmax + 1) / 2;
  const int threads = ((pairs * kJ64Lanes + 31) / 32) * 32;
  if (bmax <= 64)
    svd_jacobi_f64_kernel<4><<<njobs, threads, svd64_smem(bmax), stream>>>(jobs, bases, status);
  else
    svd_jacobi_f64_kernel<kJ64Chunks><<<njobs, threads, svd64_smem(bmax), stream>>>(jobs, bases, status);
}

int ttm64_tiles(int64_t fibres) { return (int)((fibres + kTtmF - 1) / kTtmF); }

void launch_ttm_f64(const TtmJob* jobs, int njobs, int total_tiles, int max_cols, int bmax, const Bases& bases,
                    cudaStream_t stream) {
  // shared memory sized for the plan's widest basis (the kernel pads b and the columns it uses)
  const size_t smem = ttm64_smem(bmax);
  switch ((max_cols + 15) / 16) {
    case 1: ttm_f64_kernel<1><<<total_tiles, kTtmThreads, smem, stream>>>(jobs, njobs, bases); break;
    case 2: ttm_f64_kernel<2><<<total_tiles, kTtmThreads, smem, stream>>>(jobs, njobs, bases); break;
    case 3: ttm_f64_kernel<3><<<total_tiles, kTtmThreads, smem, stream>>>(jobs, njobs, bases); break;
    case 4: ttm_f64_kernel<4><<<total_tiles, kTtmThreads, smem, stream>>>(jobs, njobs, bases); break;
    case 5: ttm_f64_kernel<5><<<total_tiles, kTtmThreads, smem, stream>>>(jobs, njobs, bases); break;
    default: ttm_f64_kernel<6><<<total_tiles, kTtmThreads, smem, stream>>>(jobs, njobs, bases); break;
  }
}

void launch_chol_step(const CholJob* jobs, int njobs, const Bases& bases, Status* status, cudaStream_t stream) {
  chol_step_kernel<<<njobs, kCholThreads, kCholSmem, stream>>>(jobs, bases, status);
}

}  // namespace tks

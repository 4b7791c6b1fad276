// Fused projection of order-3 problems (mixed-precision path): the two small contractions on the
// CUDA cores in float32, the large one on the tcgen05 tensor cores.
//
// Sec. 3.3: the projected core is H = sum_k G_k x_1 A_1k x_2 A_2k x_3 A_3k with A_nk = Q_n^T U_k^(n)
// (b_n x r_kn).  One CTA owns kRows consecutive mode-1 rows a0 of H for one problem and all of
// its a1 < b1 <= 64 and a2 < b2 <= 64, and streams the terms through shared memory in chunks of
// at most 16 mode-3 indices i2:
//   s1  W1[x, i1, i2] = sum_i0 A_1k[x0 + x, i0] G_k[i0, i1, i2]        (alpha_k folded into A_1k)
//   s2  W2[(a1, x), i2] = sum_i1 A_2k[a1, i1] W1[x, i1, i2]
//   s3  H[(a1, x), a2] += sum_i2 W2[(a1, x), i2] A_3k[a2, i2]
// s3 is the dominant contraction (2 kRows b1 b2 r_k3 flops per term): a 256 x 64 x 16 matrix
// product per chunk.  s2 writes W2, and the chunk's rows of A_3k are written, as three bfloat16
// planes each (hi + mid + lo carries the float32 value to about 2^-24); one elected thread issues
// tcgen05.mma for the plane pairs whose products reach 2^-16 relative (hi x hi into one TMEM
// accumulator, hi x mid, mid x hi, mid x mid, hi x lo, lo x hi into a second one, so that the
// large accumulator takes one rounding per chunk).  The accumulators stay in TMEM over all terms
// of the problem, so neither the per-term products nor their concatenation reach global memory;
// the epilogue reads them back with tcgen05.ld.  Every wait is bounded: on a timeout the kernel
// records TKS_ETIMEOUT, waits (bounded) for its products in flight, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bf16.cuh"
#include "fastdiv.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace tks {

namespace {

constexpr int kRows = kProj3Rows;          // mode-1 rows per CTA
constexpr int kPad = 64;                   // b2, b3 padded to 64 (N of the product)
constexpr int kChunk = kProj3Chunk;        // mode-3 indices per chunk (at most) = K of one MMA
constexpr int kGBytes = kProj3SliceBytes;  // bytes of the core slice per chunk (at most)
constexpr int kGBuf = kGBytes + 32;        // + room for the 16-byte realignment of the slice
constexpr int kW1 = kProj3W1Floats;        // floats of W1 per chunk (at most)
constexpr int kThreads = 256;
constexpr int kR = TKS_MAX_RANK;
// bf16 operand planes of s3, K-major without swizzle: core matrices of 8 rows x 8 k (16 bytes a
// row), the two of an 8-row group (k < 8, k >= 8) kLbo bytes apart, row groups kSbo bytes apart.
// The 16 spare bytes after each core matrix put the 2-byte stores of s2 on distinct banks.
constexpr int kLbo = 144;
constexpr int kSbo = 288;
constexpr int kPlaneA = 16 * kSbo;         // one M-half (128 rows (a1, x)) of one plane of W2
constexpr int kPlaneB = 8 * kSbo;          // the 64 rows a2 of one plane of A_3k
constexpr int kLd3 = 20;                   // row stride of A3 (floats): conflict-free 16-byte reads of 8 rows
constexpr int kTmemCols = 256;             // [hi x hi | corrections] x [M-half 0 | M-half 1] x 64
constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// No "memory" clobber on the copies themselves: their destinations are read only after
// cp_async_wait_all (which has one) and a barrier, and a clobber here would make the compiler
// reload every job field from global memory after each copy.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Shared-memory layout; the per-term operands A1, A2 are double-buffered by term parity, the
// per-chunk operands G, A3 by chunk parity.
struct Smem {
  unsigned char PA[3][2][kPlaneA];  // bf16 planes of W2 [plane][M-half], rows (a1, x) = 4 a1 + x
  unsigned char PB[3][kPlaneB];     // bf16 planes of the chunk's A_3k [plane], rows a2
  float A1[2][kR * kRows];          // [i0][x]
  float A2[2][kPad * kR];           // [a1][i1], row stride (r1 + 3) & ~3
  float A3[2][kPad * kLd3];         // [a2][i2c]
  float W1[kW1];                    // [i2c][i1][x], i2c stride (r1 | 1) kRows
  __align__(16) unsigned char G[2][kGBuf];   // core slice G[:, :, c0 : c0 + nc], realigned to 16 bytes
  uint64_t mma_done;                // one phase per chunk: its products have completed
  uint32_t tmem_base;
  int err;
};

__device__ __forceinline__ float core_value(uint16_t h) { return bf16_float(h); }
__device__ __forceinline__ float core_value(float v) { return v; }

struct Pos {
  int k, c;   // term, chunk of the term
};

// Chunk c of a term covers mode-3 indices [c0, c0 + nc) (the chunk length comes with the term).
__device__ __forceinline__ void chunk_range(const Proj3Term& T, const Pos& p, int& c0, int& nc) {
  c0 = p.c * T.chunk;
  nc = min(T.chunk, T.r[2] - c0);
}

// The job's fields as registers.
struct JobRegs {
  const float* AT[3];
  int64_t R[3];
  int64_t hs1, hs2;
  int b[3];
  int x0, rows;
};

// Issue the asynchronous copies of one chunk (and, on its first chunk, of the term's A1 and A2)
// into buffer `buf`; returns the element shift of the core slice inside its buffer.
template <typename CoreT>
__device__ __forceinline__ int issue_chunk(Smem& S, const JobRegs& J, const Proj3Term& T, const Pos& p, int buf,
                                           const Bases& bases) {
  const int tid = threadIdx.x;
  const int r0 = T.r[0], r1 = T.r[1];
  int c0, nc;
  chunk_range(T, p, c0, nc);
  // (the index maps below use shifts and masks only: a division by a rank costs ~20 instructions)
  if (p.c == 0) {
    const float* AT0 = J.AT[0] + T.roff[0];
    const float* AT1 = J.AT[1] + T.roff[1];
    float* A1 = S.A1[p.k & 1];
    float* A2 = S.A2[p.k & 1];
    // A1[i0][x] = A_1k[x0 + x, i0], e = kRows i0 + x
    for (int e = tid; e < r0 * kRows; e += kThreads) {
      const int x = e & (kRows - 1), i0 = e / kRows;
      if (x < J.rows) cp_async4(A1 + e, AT0 + i0 + J.R[0] * (J.x0 + x));
    }
    // A2[a1][i1] = A_2k[a1, i1]: lanes along i1, contiguous in A_2^T and in shared memory
    const int ld2 = (r1 + 3) & ~3;
    for (int e = tid; e < 32 * J.b[1]; e += kThreads) {
      const int a1 = e >> 5;
      const float* src = AT1 + J.R[1] * a1;
      for (int i1 = e & 31; i1 < r1; i1 += 32) cp_async4(A2 + a1 * ld2 + i1, src + i1);
    }
  }
  // A3[a2][i2c] = A_3k[a2, c0 + i2c]: lanes along i2c
  const float* AT2 = J.AT[2] + T.roff[2] + c0;
  float* A3 = S.A3[buf];
  for (int e = tid; e < kChunk * J.b[2]; e += kThreads) {
    const int i2c = e & (kChunk - 1), a2 = e / kChunk;
    if (i2c < nc) cp_async4(A3 + a2 * kLd3 + i2c, AT2 + i2c + J.R[2] * a2);
  }
  // the slice is contiguous: copy the 16-byte blocks that cover it (they lie in the pages of the
  // slice's own first and last bytes, so nothing outside mapped memory is touched)
  const char* g = reinterpret_cast<const char*>(at<CoreT>(bases, T.core) + (int64_t)r0 * r1 * c0);
  const char* g16 = reinterpret_cast<const char*>(reinterpret_cast<uintptr_t>(g) & ~uintptr_t(15));
  const int shift = (int)(g - g16) / (int)sizeof(CoreT);
  const int blocks = ((int)sizeof(CoreT) * (shift + r0 * r1 * nc) + 15) / 16;
  for (int e = tid; e < blocks; e += kThreads) cp_async16(S.G[buf] + 16 * e, g16 + 16 * e);
  cp_async_commit();
  return shift;
}

__device__ __forceinline__ bool advance(const Proj3Term* terms, int nterms, Pos& p) {
  if (++p.c * terms[p.k].chunk < terms[p.k].r[2]) return true;
  p.c = 0;
  return ++p.k < nterms;
}

// Byte offset of element (row, k) in a plane: row group, k block, row in the group, k in the block.
__device__ __forceinline__ int plane_offset(int row, int k) {
  return (row >> 3) * kSbo + (k >> 3) * kLbo + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t plane_desc(const void* p) {
  return tc::plain_kmajor_desc(tc::smem_u32(p), kLbo, kSbo);
}

__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

template <typename CoreT>
__global__ void __launch_bounds__(kThreads, 2) project3_kernel(const Proj3Job* __restrict__ jobs, int njobs,
                                                                Bases bases, Status* status) {
  extern __shared__ __align__(16) unsigned char p3raw[];
  Smem& S = *reinterpret_cast<Smem*>(p3raw);
  volatile int* err = &S.err;
  const Proj3Job& Jg = jobs[blockIdx.x];
  const Proj3Term* terms = reinterpret_cast<const Proj3Term*>(jobs + njobs) + Jg.term_begin;
  const int nterms = Jg.nterms;
  JobRegs J;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    J.AT[q] = at<float>(bases, Jg.AT[q]);
    J.R[q] = Jg.R[q];
    J.b[q] = Jg.b[q];
  }
  J.x0 = Jg.x0;
  J.rows = Jg.rows;
  J.hs1 = Jg.hs1;
  J.hs2 = Jg.hs2;
  double* const Hout = at<double>(bases, Jg.H);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b1 = J.b[1], b2 = J.b[2];
  const bool two_halves = b1 > 32;   // M-half 1 holds the rows of a1 >= 32

  // rows x >= J.rows of A1 stay zero (never copied into), so their rows of W2 are zero
  for (int e = tid; e < 2 * kR * kRows; e += kThreads) (&S.A1[0][0])[e] = 0.f;
  if (tid == 0) {
    tc::mbar_init(&S.mma_done, 1);
    *err = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc(&S.tmem_base, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();   // the zero fill lands before any copy into A1; the barrier and TMEM are set up
  tc::fence_after_sync();
  const uint32_t tmem = S.tmem_base;
  int issued = 0;   // chunks whose products were issued

  if (nterms > 0) {
    Pos cur{0, 0};
    int shift = issue_chunk<CoreT>(S, J, terms[0], cur, 0, bases);
    int buf = 0;
    bool more = true;
    while (more) {
      const Proj3Term& T = terms[cur.k];
      const int r0 = T.r[0], r1 = T.r[1], r1s = r1 | 1;
      int c0, nc;
      chunk_range(T, cur, c0, nc);
      cp_async_wait_all();
      __syncthreads();   // this chunk is in shared memory; every thread is done with the other buffers
      Pos nxt = cur;
      more = advance(terms, nterms, nxt);
      int next_shift = 0;
      if (more) next_shift = issue_chunk<CoreT>(S, J, terms[nxt.k], nxt, buf ^ 1, bases);
      const float alpha = T.alpha;
      const float* A1 = S.A1[cur.k & 1];
      const float* A2 = S.A2[cur.k & 1];
      const float* A3 = S.A3[buf];
      const CoreT* Gs = reinterpret_cast<const CoreT*>(S.G[buf]) + shift;
      // s1: pair p = i1 + r1 i2c reads the contiguous core column G[:, i1, c0 + i2c]
      const SmallDiv dr1(r1);
      for (int p = tid; p < nc * r1; p += kThreads) {
        const int i2c = dr1.quo(p), i1 = p - i2c * r1;
        const CoreT* g = Gs + r0 * p;
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i0 = 0; i0 < r0; ++i0) {
          const float gv = core_value(g[i0]);
          const float4 a = *reinterpret_cast<const float4*>(A1 + kRows * i0);
          w.x = fmaf(a.x, gv, w.x);
          w.y = fmaf(a.y, gv, w.y);
          w.z = fmaf(a.z, gv, w.z);
          w.w = fmaf(a.w, gv, w.w);
        }
        *reinterpret_cast<float4*>(S.W1 + kRows * (i2c * r1s + i1)) =
            make_float4(alpha * w.x, alpha * w.y, alpha * w.z, alpha * w.w);
      }
      // the planes are free once the products of the previous chunk have completed
      if (issued > 0 && !tc::mbar_wait(&S.mma_done, (issued - 1) & 1, kWaitCycles)) *err = 1;
      __syncthreads();
      // s2: a thread owns a1 = a1b .. a1b + 3 and x = 0..3 of one i2c and writes them, split, to
      // column k = i2c of the W2 planes (zeros for i2c >= nc: the product runs over k < 16);
      // rows a1 >= b1 only reach rows of the product that are never read
      {
        const int i2c = tid & 15, a1b = (tid >> 4) * 4;
        if (a1b < b1) {
          float w2[4][kRows];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int x = 0; x < kRows; ++x) w2[j][x] = 0.f;
          if (i2c < nc) {
            const float* w1 = S.W1 + kRows * (i2c * r1s);
            const int ld2 = (r1 + 3) & ~3;
            const float* a2r = A2 + a1b * ld2;   // rows a1b .. a1b + 3
            int i1 = 0;
            for (; i1 + 4 <= r1; i1 += 4) {   // four i1 at a time: 16-byte reads along i1
              float4 a[4], w[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) a[j] = *reinterpret_cast<const float4*>(a2r + j * ld2 + i1);
#pragma unroll
              for (int u = 0; u < 4; ++u) w[u] = *reinterpret_cast<const float4*>(w1 + kRows * (i1 + u));
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float av[4] = {a[j].x, a[j].y, a[j].z, a[j].w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  w2[j][0] = fmaf(av[u], w[u].x, w2[j][0]);
                  w2[j][1] = fmaf(av[u], w[u].y, w2[j][1]);
                  w2[j][2] = fmaf(av[u], w[u].z, w2[j][2]);
                  w2[j][3] = fmaf(av[u], w[u].w, w2[j][3]);
                }
              }
            }
            for (; i1 < r1; ++i1) {
              const float4 w = *reinterpret_cast<const float4*>(w1 + kRows * i1);
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float av = a2r[j * ld2 + i1];
                w2[j][0] = fmaf(av, w.x, w2[j][0]);
                w2[j][1] = fmaf(av, w.y, w2[j][1]);
                w2[j][2] = fmaf(av, w.z, w2[j][2]);
                w2[j][3] = fmaf(av, w.w, w2[j][3]);
              }
            }
          }
          const int half = a1b >> 5;   // rows 4 a1b .. 4 a1b + 15 lie in one M-half
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int x = 0; x < kRows; ++x) {
              const int off = plane_offset((4 * (a1b + j) + x) & 127, i2c);
              uint16_t h0, h1, h2;
              split3(w2[j][x], h0, h1, h2);
              *reinterpret_cast<uint16_t*>(S.PA[0][half] + off) = h0;
              *reinterpret_cast<uint16_t*>(S.PA[1][half] + off) = h1;
              *reinterpret_cast<uint16_t*>(S.PA[2][half] + off) = h2;
            }
        }
      }
      // rows a2 < b2 of the chunk's A_3k, split, k = i2c (zeros for i2c >= nc)
      if (tid < 2 * kPad && (tid & (kPad - 1)) < b2) {
        const int a2 = tid & (kPad - 1), kb = tid >> 6;
        const float4 lo = *reinterpret_cast<const float4*>(A3 + a2 * kLd3 + 8 * kb);
        const float4 hi = *reinterpret_cast<const float4*>(A3 + a2 * kLd3 + 8 * kb + 4);
        const float av[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        uint32_t q0[4], q1[4], q2[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 8 * kb + 2 * e;
          const float v0 = k < nc ? av[2 * e] : 0.f;
          const float v1 = k + 1 < nc ? av[2 * e + 1] : 0.f;
          uint16_t l0, l1, l2, u0, u1, u2;
          split3(v0, l0, l1, l2);
          split3(v1, u0, u1, u2);
          q0[e] = pack2(l0, u0);
          q1[e] = pack2(l1, u1);
          q2[e] = pack2(l2, u2);
        }
        const int off = plane_offset(a2, 8 * kb);
        *reinterpret_cast<uint4*>(S.PB[0] + off) = make_uint4(q0[0], q0[1], q0[2], q0[3]);
        *reinterpret_cast<uint4*>(S.PB[1] + off) = make_uint4(q1[0], q1[1], q1[2], q1[3]);
        *reinterpret_cast<uint4*>(S.PB[2] + off) = make_uint4(q2[0], q2[1], q2[2], q2[3]);
      }
      tc::fence_proxy_async_smem();
      __syncthreads();   // the planes are complete
      if (*err) break;   // read after the barrier: the same decision in every thread
      // s3 on the tensor cores
      if (tid == 0) {
        tc::fence_after_sync();
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kPad);
        const uint64_t db0 = plane_desc(S.PB[0]), db1 = plane_desc(S.PB[1]), db2 = plane_desc(S.PB[2]);
        const uint32_t first = issued > 0 ? 1u : 0u;
        for (int h = 0; h < (two_halves ? 2 : 1); ++h) {
          const uint64_t da0 = plane_desc(S.PA[0][h]), da1 = plane_desc(S.PA[1][h]), da2 = plane_desc(S.PA[2][h]);
          const uint32_t big = tmem + (uint32_t)(kPad * h), corr = tmem + (uint32_t)(2 * kPad + kPad * h);
          tc::mma_bf16(big, da0, db0, idesc, first);
          tc::mma_bf16(corr, da0, db1, idesc, first);
          tc::mma_bf16(corr, da1, db0, idesc, 1u);
          tc::mma_bf16(corr, da1, db1, idesc, 1u);
          tc::mma_bf16(corr, da0, db2, idesc, 1u);
          tc::mma_bf16(corr, da2, db0, idesc, 1u);
        }
        tc::mma_commit(&S.mma_done);
      }
      ++issued;
      cur = nxt;
      shift = next_shift;
      buf ^= 1;
    }
  }
  cp_async_wait_all();   // copies of a chunk that an error left unconsumed

  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows m of an M-half) and columns
  // 32 (w / 4) .. + 31 (a2); row m of M-half h is a1 = 32 h + m / 4, x = m % 4
  const bool done = issued == 0 || tc::mbar_wait(&S.mma_done, (issued - 1) & 1, kWaitCycles);
  const bool good = __all_sync(0xffffffffu, done && !*err);   // one decision per warp (tcgen05.ld is warp-wide)
  tc::fence_after_sync();
  if (!good && lane == 0) *err = 1;
  if (good) {
    const int q = warp & 3, cb = 32 * (warp >> 2);
    const int m = 32 * q + lane, x = m & 3;
    for (int h = 0; h < (two_halves ? 2 : 1); ++h) {
      float sum[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) sum[j] = 0.f;
      if (issued > 0) {
        uint32_t r[32];
        const uint32_t row_addr = tmem + ((uint32_t)(32 * q) << 16);
        tc::tmem_ld32(row_addr + (uint32_t)(kPad * h + cb), r);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[j] = __uint_as_float(r[j]);
        tc::tmem_ld32(row_addr + (uint32_t)(2 * kPad + kPad * h + cb), r);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[j] += __uint_as_float(r[j]);
      }
      const int a1 = 32 * h + (m >> 2);
      if (a1 < b1 && x < J.rows) {
        double* dst = Hout + J.x0 + x + J.hs1 * a1 + J.hs2 * cb;
        const int ncol = min(32, b2 - cb);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j < ncol) *dst = f32_to_f64_exact(sum[j]);
          dst += J.hs2;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
  if (tid == 0 && *err && status) atomicCAS(&status->code, 0, (int)TKS_ETIMEOUT);
}

constexpr size_t kSmemBytes = sizeof(Smem);
static_assert(kSmemBytes <= 112 * 1024, "two CTAs per SM");

// ----------------------------------------------------------------------------- order-4 fold
// G'_k(a1)[i0, i2, i3] = alpha_k sum_i1 A_2k[a1, i1] G_k[i0, i1, i2, i3] for one i3 and all a1:
// the slice G_k[:, :, :, i3] and the rows of A_2k go to shared memory; a thread forms outputs
// (i0, i2, a1) with i0 fastest, so the writes run along the output's contiguous index.
__global__ void __launch_bounds__(256) fold4_kernel(const Fold4Job* __restrict__ jobs, Bases bases) {
  extern __shared__ __align__(16) float f4s[];
  const Fold4Job& J = jobs[blockIdx.x];
  const int r0 = J.r[0], r1 = J.r[1], r2 = J.r[2], r3 = J.r[3], b1 = J.b1, i3 = J.i3;
  const int slice = r0 * r1 * r2;
  float* A2 = f4s;                 // [a1][i1]
  float* Gs = A2 + b1 * r1;        // [i0 + r0 (i1 + r1 i2)]
  const uint16_t* G = at<uint16_t>(bases, J.core) + (int64_t)slice * i3;
  const float* AT1 = at<float>(bases, J.AT1) + J.roff1;
  const float alpha = J.alpha;
  for (int e = threadIdx.x; e < b1 * r1; e += blockDim.x) {
    const int i1 = e % r1, a1 = e / r1;
    A2[a1 * r1 + i1] = alpha * AT1[i1 + J.R1 * a1];
  }
  for (int e = threadIdx.x; e < slice; e += blockDim.x) Gs[e] = bf16_float(G[e]);
  __syncthreads();
  float* out = at<float>(bases, J.out);
  const int64_t blk = (int64_t)r0 * r2 * r3;
  const int per_a1 = r0 * r2;
  for (int e = threadIdx.x; e < b1 * per_a1; e += blockDim.x) {
    const int a1 = e / per_a1, rem = e - a1 * per_a1;
    const int i0 = rem % r0, i2 = rem / r0;
    const float* g = Gs + i0 + r0 * r1 * i2;
    const float* a = A2 + a1 * r1;
    float v = 0.f;
    for (int i1 = 0; i1 < r1; ++i1) v = fmaf(a[i1], g[r0 * i1], v);
    out[blk * a1 + i0 + (int64_t)r0 * (i2 + (int64_t)r2 * i3)] = v;
  }
}

}  // namespace

size_t proj3_smem_bytes() { return kSmemBytes; }

cudaError_t prepare_proj3() {
  cudaError_t e =
      cudaFuncSetAttribute(project3_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(project3_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

size_t fold4_smem_bytes(int r0, int r1, int r2, int b1) {
  return sizeof(float) * ((size_t)b1 * r1 + (size_t)r0 * r1 * r2);
}

cudaError_t prepare_fold4() {
  return cudaFuncSetAttribute(fold4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void launch_fold4(const Fold4Job* jobs, int njobs, size_t smem, const Bases& bases, cudaStream_t stream) {
  fold4_kernel<<<njobs, 256, smem, stream>>>(jobs, bases);
}

void launch_proj3(const Proj3Job* jobs, int njobs, bool f32_cores, const Bases& bases, Status* status,
                  cudaStream_t stream) {
  if (f32_cores)
    project3_kernel<float><<<njobs, kThreads, kSmemBytes, stream>>>(jobs, njobs, bases, status);
  else
    project3_kernel<uint16_t><<<njobs, kThreads, kSmemBytes, stream>>>(jobs, njobs, bases, status);
}

}  // namespace tks

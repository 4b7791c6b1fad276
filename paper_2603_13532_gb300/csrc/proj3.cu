// Fused projection of order-3 problems (mixed-precision path): the first mode product on the CUDA
// cores in float32, the second and the third on the tcgen05 tensor cores.
//
// Sec. 3.3: the projected core is H = sum_k G_k x_1 A_1k x_2 A_2k x_3 A_3k with A_nk = Q_n^T U_k^(n)
// (b_n x r_kn).  One CTA owns kRows consecutive mode-1 rows a0 of H for one problem and all of
// its a1 < b1 <= 64 and a2 < b2 <= 64, and streams the terms through shared memory in chunks of
// at most 16 mode-3 indices i2:
//   s1  W1[x, i1, i2] = alpha_k sum_i0 A_1k[x0 + x, i0] G_k[i0, i1, i2]       (CUDA cores)
//   s2  W2[a1, (x, i2)] = sum_i1 A_2k[a1, i1] W1[x, i1, i2]                  (tensor cores)
//   s3  H[(a1, x), a2] += sum_i2 W2[(a1, x), i2] A_3k[a2, i2]                 (tensor cores)
// Every tensor-core operand is a float32 matrix split exactly into three bfloat16 planes (hi + mid
// + lo = the value; hi and mid are the leading 8 significant bits of the value and of the
// remainder), and a product takes the six plane pairs whose terms reach 2^-24 relative (hi x hi,
// hi x mid, mid x hi, mid x mid, hi x lo, lo x hi).  s1 writes W1 straight into the planes of s2's
// B operand (rows 16 x + i2, k = i1); A_2k's planes (rows a1, k = i1; an M = 128 product with rows
// a1 < 64) are formed once per term.  s2 lands in TMEM (lane a1, column 16 x + i2); four warps read
// it back and write it, split, as the planes of s3's A operand (rows 4 a1 + x, k = i2) with 16-byte
// stores.  s3 accumulates H over all terms of the problem in TMEM (two M-halves of 128 rows (a1, x),
// 64 columns each); the epilogue reads it back with tcgen05.ld.  Every wait is bounded: on a
// timeout the kernel records TKS_ETIMEOUT, waits (bounded) for its products in flight, frees TMEM
// and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bf16.cuh"
#include "fastdiv.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace tks {

namespace {

constexpr int kRows = kProj3Rows;          // mode-1 rows per CTA (4)
constexpr int kPad = 64;                   // b2, b3 padded to 64
constexpr int kChunk = kProj3Chunk;        // mode-3 indices per chunk (at most) = K of s3
constexpr int kGBytes = kProj3SliceBytes;  // bytes of the core slice per chunk (at most)
constexpr int kGBuf = kGBytes + 32;        // + room for the 16-byte realignment of the slice
constexpr int kThreads = 256;
constexpr int kR = TKS_MAX_RANK;
constexpr int kLbo = 128;                  // K-major tiles without swizzle: k blocks 128 bytes apart
// s2 operands (K = kp1 <= 64): k blocks 144 bytes apart (the 2-byte stores of W1, consecutive k
// across a warp, fall on distinct banks), 8-row groups kp1 / 8 * 144 bytes apart
constexpr int kLbo2 = 144;
// s3 operands (K = 16): 8-row groups 272 bytes apart (256 + 16, so that the 16-byte stores of a
// warp spread over the banks)
constexpr int kSbo3 = 272;
constexpr int kPlaneA3 = 16 * kSbo3;       // one M-half (128 rows (a1, x)) of one plane of W2
constexpr int kPlaneB3 = 8 * kSbo3;        // the 64 rows a2 of one plane of A_3k
constexpr int kLd3 = 20;                   // row stride of the staged A_3k chunk (floats)
constexpr int kTmemCols = 256;             // H: [M-half 0 | M-half 1] x 64; s2: 64 columns from 128
constexpr int kS2Col = 2 * kPad;
constexpr long long kWaitCycles = 4000000000LL;   // about 2 s at 2 GHz

// Shared-memory layout for kp1max = the largest r_1 of the launch rounded up to 16 (K of s2).
struct Layout {
  int a2p, w1p, pa, pb, a1f, a2f, a3f, g, bars, total;
  int plane2;   // bytes of one s2 plane slot: 64 rows x kp1max k
};
__host__ __device__ inline Layout proj3_layout(int kp1max) {
  Layout L;
  L.plane2 = 8 * (kp1max / 8) * kLbo2;
  L.a2p = 0;                                   // 3 planes of A_2k (an M = 128 product reads on
  L.w1p = L.a2p + 3 * L.plane2;                // into the next slot: the last one into W1's)
  L.pa = L.w1p + 3 * L.plane2;                 // 3 planes of W1
  L.pb = L.pa + 3 * 2 * kPlaneA3;              // 3 x 2 M-halves of W2
  L.a1f = L.pb + 3 * kPlaneB3;                 // 3 planes of the chunk's A_3k
  L.a2f = L.a1f + 2 * kR * kRows * 4;          // A_1k rows, float32, by term parity
  L.a3f = L.a2f + 64 * kp1max * 4;             // A_2k, float32 (one term)
  L.g = L.a3f + 2 * kPad * kLd3 * 4;           // the chunk's A_3k rows, float32, by chunk parity
  L.bars = L.g + 2 * kGBuf;                    // the chunk's core slice, by chunk parity
  L.total = L.bars + 64;
  return L;
}

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

__device__ __forceinline__ float core_value(uint16_t h) { return bf16_float(h); }
__device__ __forceinline__ float core_value(float v) { return v; }

// v = hi + mid + lo exactly, each part a bfloat16 in the upper 16 bits: masks and exact float32
// subtractions, no conversion instructions.
__device__ __forceinline__ void split3_exact(float v, uint32_t& u0, uint32_t& u1, uint32_t& u2) {
  u0 = __float_as_uint(v) & 0xffff0000u;
  const float r1 = v - __uint_as_float(u0);
  u1 = __float_as_uint(r1) & 0xffff0000u;
  u2 = __float_as_uint(r1 - __uint_as_float(u1));
}
// eight values as the 16-byte rows of three planes
__device__ __forceinline__ void split3_row8(const float (&v)[8], uint4& p0, uint4& p1, uint4& p2) {
  uint32_t q0[4], q1[4], q2[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    uint32_t a0, a1, a2, b0, b1, b2;
    split3_exact(v[2 * e], a0, a1, a2);
    split3_exact(v[2 * e + 1], b0, b1, b2);
    q0[e] = __byte_perm(a0, b0, 0x7632);
    q1[e] = __byte_perm(a1, b1, 0x7632);
    q2[e] = __byte_perm(a2, b2, 0x7632);
  }
  p0 = make_uint4(q0[0], q0[1], q0[2], q0[3]);
  p1 = make_uint4(q1[0], q1[1], q1[2], q1[3]);
  p2 = make_uint4(q2[0], q2[1], q2[2], q2[3]);
}

// Byte offset of element (row, k) in a K-major plane: k blocks lbo bytes apart, 8-row groups sbo.
__device__ __forceinline__ int plane_offset(int row, int k, int sbo, int lbo = kLbo) {
  return (row >> 3) * sbo + (k >> 3) * lbo + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t plane_desc(uint32_t addr, int sbo, int lbo = kLbo) {
  return tc::plain_kmajor_desc(addr, (uint32_t)lbo, (uint32_t)sbo);
}

struct Pos {
  int k, c;   // term, chunk of the term
};

// Chunk c of a term covers mode-3 indices [c0, c0 + nc) (the chunk length comes with the term).
__device__ __forceinline__ void chunk_range(const Proj3Term& T, const Pos& p, int& c0, int& nc) {
  c0 = p.c * T.chunk;
  nc = min(T.chunk, T.r[2] - c0);
}

__device__ __forceinline__ bool advance(const Proj3Term* terms, int nterms, Pos& p) {
  if (++p.c * terms[p.k].chunk < terms[p.k].r[2]) return true;
  p.c = 0;
  return ++p.k < nterms;
}

// The job's fields as registers.
struct JobRegs {
  const float* AT[3];
  int64_t R[3];
  int64_t hs1, hs2;
  int b[3];
  int x0, rows;
};

// Asynchronous copies of one chunk into buffer `buf`: its core slice and A_3k rows, and on a term's
// first chunk the term's A_1k rows; returns the element shift of the core slice in its buffer.
template <typename CoreT>
__device__ __forceinline__ int issue_chunk(unsigned char* sm, const Layout& L, const JobRegs& J, const Proj3Term& T,
                                           const Pos& p, int buf, const Bases& bases) {
  const int tid = threadIdx.x;
  const int r0 = T.r[0], r1 = T.r[1];
  int c0, nc;
  chunk_range(T, p, c0, nc);
  if (p.c == 0) {
    // A1[i0][x] = A_1k[x0 + x, i0] (rows x >= rows stay zero: never copied into)
    const float* AT0 = J.AT[0] + T.roff[0];
    float* A1 = reinterpret_cast<float*>(sm + L.a1f) + (p.k & 1) * kR * kRows;
    for (int e = tid; e < r0 * kRows; e += kThreads) {
      const int x = e & (kRows - 1), i0 = e / kRows;
      if (x < J.rows) cp_async4(A1 + e, AT0 + i0 + J.R[0] * (J.x0 + x));
    }
  }
  // A3[a2][i2c] = A_3k[a2, c0 + i2c]
  const float* AT2 = J.AT[2] + T.roff[2] + c0;
  float* A3 = reinterpret_cast<float*>(sm + L.a3f) + buf * kPad * kLd3;
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
  unsigned char* gb = sm + L.g + buf * kGBuf;
  for (int e = tid; e < blocks; e += kThreads) cp_async16(gb + 16 * e, g16 + 16 * e);
  return shift;
}

// A2f[a1][i1] = A_2k[a1, i1] of one term (row stride (r1 + 3) & ~3).
__device__ __forceinline__ void issue_a2(unsigned char* sm, const Layout& L, const JobRegs& J, const Proj3Term& T) {
  const int r1 = T.r[1], ld2 = (r1 + 3) & ~3;
  const float* AT1 = J.AT[1] + T.roff[1];
  float* A2 = reinterpret_cast<float*>(sm + L.a2f);
  for (int e = threadIdx.x; e < 32 * J.b[1]; e += kThreads) {
    const int a1 = e >> 5;
    const float* src = AT1 + J.R[1] * a1;
    for (int i1 = e & 31; i1 < r1; i1 += 32) cp_async4(A2 + a1 * ld2 + i1, src + i1);
  }
}

template <typename CoreT>
__global__ void __launch_bounds__(kThreads, 2) project3_kernel(const Proj3Job* __restrict__ jobs, int njobs,
                                                                Bases bases, Status* status) {
  extern __shared__ __align__(16) unsigned char p3raw[];
  const Proj3Job& Jg = jobs[blockIdx.x];
  const Layout L = proj3_layout(Jg.kp1max);
  unsigned char* sm = p3raw;
  uint64_t* s2_done = reinterpret_cast<uint64_t*>(sm + L.bars);
  uint64_t* s3_done = s2_done + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(s3_done + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);
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

  // rows x >= J.rows of A1 stay zero (never copied into), so their rows of W1 are zero
  float* A1all = reinterpret_cast<float*>(sm + L.a1f);
  for (int e = tid; e < 2 * kR * kRows; e += kThreads) A1all[e] = 0.f;
  if (tid == 0) {
    tc::mbar_init(s2_done, 1);
    tc::mbar_init(s3_done, 1);
    *err = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();   // the zero fill lands before any copy into A1; the barriers and TMEM are set up
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  int issued = 0;   // chunks whose last products (s3) were issued
  int s2_issued = 0;

  if (nterms > 0) {
    Pos cur{0, 0};
    int shift = issue_chunk<CoreT>(sm, L, J, terms[0], cur, 0, bases);
    issue_a2(sm, L, J, terms[0]);
    cp_async_commit();
    int buf = 0;
    bool more = true;
    while (more) {
      const Proj3Term& T = terms[cur.k];
      const int r0 = T.r[0], r1 = T.r[1];
      const int kp1 = (r1 + 15) & ~15, sbo2 = kp1 / 8 * kLbo2;
      int c0, nc;
      chunk_range(T, cur, c0, nc);
      cp_async_wait_all();
      __syncthreads();   // this chunk is in shared memory; every thread is done with the other buffers
      Pos nxt = cur;
      more = advance(terms, nterms, nxt);
      int next_shift = 0;
      if (more) next_shift = issue_chunk<CoreT>(sm, L, J, terms[nxt.k], nxt, buf ^ 1, bases);
      cp_async_commit();
      const float alpha = T.alpha;
      const float* A1 = reinterpret_cast<const float*>(sm + L.a1f) + (cur.k & 1) * kR * kRows;
      const float* A3 = reinterpret_cast<const float*>(sm + L.a3f) + buf * kPad * kLd3;
      const CoreT* Gs = reinterpret_cast<const CoreT*>(sm + L.g + buf * kGBuf) + shift;
      unsigned char* A2p = sm + L.a2p;
      unsigned char* W1p = sm + L.w1p;
      if (cur.c == 0) {
        // the term's A_2k planes: rows a1 < 64 (zero for a1 >= b1), k = i1 < kp1 (zero for i1 >= r1)
        // (16-byte reads: the rows are ld2 = (r1 + 3) & ~3 floats apart; a read past r1 stays inside
        // the buffer and is replaced by zero)
        const float* A2 = reinterpret_cast<const float*>(sm + L.a2f);
        const int ld2 = (r1 + 3) & ~3;
        for (int item = tid; item < 64 * (kp1 / 8); item += kThreads) {
          const int a1 = item & 63, kb = item >> 6;
          const float4 lo = *reinterpret_cast<const float4*>(A2 + a1 * ld2 + 8 * kb);
          const float4 hi = *reinterpret_cast<const float4*>(A2 + a1 * ld2 + 8 * kb + 4);
          const float raw[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = (a1 < b1 && 8 * kb + e < r1) ? raw[e] : 0.f;
          uint4 p0, p1, p2;
          split3_row8(v, p0, p1, p2);
          const int off = plane_offset(a1, 8 * kb, sbo2, kLbo2);
          *reinterpret_cast<uint4*>(A2p + off) = p0;
          *reinterpret_cast<uint4*>(A2p + L.plane2 + off) = p1;
          *reinterpret_cast<uint4*>(A2p + 2 * L.plane2 + off) = p2;
        }
      }
      // s1: pair p = i1 + kp1 i2c reads the contiguous core column G[:, i1, c0 + i2c] and writes
      // its four rows x of W1, split, to rows 16 x + i2c, column i1 of the s2 planes (zeros
      // outside i1 < r1, i2c < nc; the columns i1 >= r1 only on the term's first chunk)
      {
        const SmallDiv dk(kp1);
        for (int p = tid; p < kp1 * kChunk; p += kThreads) {
          const int i2c = dk.quo(p), i1 = p - i2c * kp1;
          // columns i1 >= r1 hold zeros from the term's first chunk on
          if (i1 >= r1 && cur.c > 0) continue;
          float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
          if (i1 < r1 && i2c < nc) {
            const CoreT* g = Gs + r0 * (i1 + r1 * i2c);
            for (int i0 = 0; i0 < r0; ++i0) {
              const float gv = core_value(g[i0]);
              const float4 a = *reinterpret_cast<const float4*>(A1 + kRows * i0);
              w.x = fmaf(a.x, gv, w.x);
              w.y = fmaf(a.y, gv, w.y);
              w.z = fmaf(a.z, gv, w.z);
              w.w = fmaf(a.w, gv, w.w);
            }
          }
          const float wx[4] = {alpha * w.x, alpha * w.y, alpha * w.z, alpha * w.w};
#pragma unroll
          for (int x = 0; x < kRows; ++x) {
            uint32_t u0, u1, u2;
            split3_exact(wx[x], u0, u1, u2);
            const int off = plane_offset(16 * x + i2c, i1, sbo2, kLbo2);
            *reinterpret_cast<uint16_t*>(W1p + off) = (uint16_t)(u0 >> 16);
            *reinterpret_cast<uint16_t*>(W1p + L.plane2 + off) = (uint16_t)(u1 >> 16);
            *reinterpret_cast<uint16_t*>(W1p + 2 * L.plane2 + off) = (uint16_t)(u2 >> 16);
          }
        }
      }
      // the planes of s3 are free once the products of the previous chunk have completed
      if (issued > 0 && !tc::mbar_wait(s3_done, (issued - 1) & 1, kWaitCycles)) *err = 1;
      // the chunk's A_3k planes: rows a2 < 64 (zero for a2 >= b2), k = i2c < 16 (zero for i2c >= nc)
      if (tid < 2 * kPad) {
        const int a2 = tid & (kPad - 1), kb = tid >> 6;
        const float4 lo = *reinterpret_cast<const float4*>(A3 + a2 * kLd3 + 8 * kb);
        const float4 hi = *reinterpret_cast<const float4*>(A3 + a2 * kLd3 + 8 * kb + 4);
        const float raw[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = (a2 < b2 && 8 * kb + e < nc) ? raw[e] : 0.f;
        uint4 p0, p1, p2;
        split3_row8(v, p0, p1, p2);
        unsigned char* PB = sm + L.pb;
        const int off = plane_offset(a2, 8 * kb, kSbo3);
        *reinterpret_cast<uint4*>(PB + off) = p0;
        *reinterpret_cast<uint4*>(PB + kPlaneB3 + off) = p1;
        *reinterpret_cast<uint4*>(PB + 2 * kPlaneB3 + off) = p2;
      }
      tc::fence_proxy_async_smem();
      __syncthreads();   // A_2k, W1 and A_3k planes complete
      if (*err) break;   // read after the barrier: the same decision in every thread
      // s2 on the tensor cores: D2[a1, 16 x + i2c] over k = i1 < kp1
      if (tid == 0) {
        tc::fence_after_sync();
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kPad);
        const uint32_t a0 = smem_addr(A2p), w0 = smem_addr(W1p);
        const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};
        for (int ks = 0; ks < kp1 / 16; ++ks)
#pragma unroll
          for (int u = 0; u < 6; ++u)
            tc::mma_bf16(tmem + (uint32_t)kS2Col, plane_desc(a0 + pa[u] * L.plane2 + 2 * kLbo2 * ks, sbo2, kLbo2),
                         plane_desc(w0 + pb[u] * L.plane2 + 2 * kLbo2 * ks, sbo2, kLbo2), idesc,
                         (ks > 0 || u > 0) ? 1u : 0u);
        tc::mma_commit(s2_done);
      }
      ++s2_issued;
      // the next term's A_2k rows, once this term's planes are formed (every term's first chunk
      // forms them before the barrier above)
      if (more && nxt.c == 0) {
        issue_a2(sm, L, J, terms[nxt.k]);
        cp_async_commit();
      }
      // s2 read back by warps 0, 1, 4, 5 (TMEM lanes a1 = 0..63; columns x = 0, 1 or 2, 3), split
      // and written as rows 4 a1 + x of the W2 planes
      const int q = warp & 3;
      if (q < 2) {
        const bool done = tc::mbar_wait(s2_done, issued & 1, kWaitCycles);
        if (!__all_sync(0xffffffffu, done)) {
          if (lane == 0) *err = 1;
        } else {
          tc::fence_after_sync();
          const int xh = warp >> 2;   // columns 32 xh .. 32 xh + 31: x = 2 xh, 2 xh + 1
          uint32_t v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kS2Col + 32 * xh), v);
          tc::tmem_ld_wait();
          const int a1 = 32 * q + lane;
          unsigned char* PA = sm + L.pa;
#pragma unroll
          for (int xx = 0; xx < 2; ++xx) {
            const int row = 4 * a1 + 2 * xh + xx;     // < 256
            const int half = row >> 7, rr = row & 127;
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) {
              float f[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) f[e] = __uint_as_float(v[16 * xx + 8 * kb + e]);
              uint4 p0, p1, p2;
              split3_row8(f, p0, p1, p2);
              const int off = half * kPlaneA3 + plane_offset(rr, 8 * kb, kSbo3);
              *reinterpret_cast<uint4*>(PA + off) = p0;
              *reinterpret_cast<uint4*>(PA + 2 * kPlaneA3 + off) = p1;
              *reinterpret_cast<uint4*>(PA + 4 * kPlaneA3 + off) = p2;
            }
          }
        }
      }
      tc::fence_proxy_async_smem();
      tc::fence_before_sync();
      __syncthreads();   // the W2 planes are complete
      if (*err) break;
      // s3 on the tensor cores: H[(a1, x), a2] += W2 A_3k^T, the six plane pairs per M-half
      if (tid == 0) {
        tc::fence_after_sync();
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kPad);
        const uint32_t pa0 = smem_addr(sm + L.pa), pb0 = smem_addr(sm + L.pb);
        const int qa[6] = {0, 0, 1, 1, 0, 2}, qb[6] = {0, 1, 0, 1, 2, 0};
        for (int h = 0; h < (two_halves ? 2 : 1); ++h)
#pragma unroll
          for (int u = 0; u < 6; ++u)
            tc::mma_bf16(tmem + (uint32_t)(kPad * h),
                         plane_desc(pa0 + (2 * qa[u] + h) * kPlaneA3, kSbo3), plane_desc(pb0 + qb[u] * kPlaneB3, kSbo3),
                         idesc, (issued > 0 || u > 0) ? 1u : 0u);
        tc::mma_commit(s3_done);
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
  const bool done = issued == 0 || tc::mbar_wait(s3_done, (issued - 1) & 1, kWaitCycles);
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
        tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kPad * h + cb), r);
        tc::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[j] = __uint_as_float(r[j]);
      }
      const int a1 = 32 * h + (m >> 2);
      if (a1 < b1 && x < J.rows) {
        double* dst = Hout + J.x0 + x + J.hs1 * a1 + J.hs2 * cb;
        const int ncol = min(32, b2 - cb);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (j < ncol) *dst = (double)sum[j];
          dst += J.hs2;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  // after a timeout, the products issued last complete before TMEM is freed (bounded)
  if (*err && tid == 0) {
    if (s2_issued > 0) tc::mbar_wait(s2_done, (s2_issued - 1) & 1, kWaitCycles);
    if (issued > 0) tc::mbar_wait(s3_done, (issued - 1) & 1, kWaitCycles);
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
  if (tid == 0 && *err && status) atomicCAS(&status->code, 0, (int)TKS_ETIMEOUT);
}

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

size_t proj3_smem_bytes(int kp1max) { return (size_t)proj3_layout(kp1max).total; }

cudaError_t prepare_proj3() {
  const int most = (int)proj3_smem_bytes(kR);
  cudaError_t e = cudaFuncSetAttribute(project3_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(project3_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
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

void launch_proj3(const Proj3Job* jobs, int njobs, size_t smem, bool f32_cores, const Bases& bases, Status* status,
                  cudaStream_t stream) {
  if (f32_cores)
    project3_kernel<float><<<njobs, kThreads, smem, stream>>>(jobs, njobs, bases, status);
  else
    project3_kernel<uint16_t><<<njobs, kThreads, smem, stream>>>(jobs, njobs, bases, status);
}

}  // namespace tks

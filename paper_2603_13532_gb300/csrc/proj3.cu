// Fused projection of order-3 problems on the CUDA cores, in float32 (mixed-precision path).
//
// Sec. 3.3: the projected core is H = sum_k G_k x_1 A_1k x_2 A_2k x_3 A_3k with A_nk = Q_n^T U_k^(n)
// (b_n x r_kn).  One CTA owns kRows consecutive mode-1 rows a0 of H for one problem and all of
// its a1 < b1 <= 64 and a2 < b2 <= 64, holds that block of H in registers, and streams the terms
// through shared memory in chunks of mode-3 indices i2:
//   s1  W1[x, i1, i2] = sum_i0 A_1k[x0 + x, i0] G_k[i0, i1, i2]        (alpha_k folded into A_1k)
//   s2  W2[a1, x, i2] = sum_i1 A_2k[a1, i1] W1[x, i1, i2]
//   s3  H[x, a1, a2] += sum_i2 W2[a1, x, i2] A_3k[a2, i2]
// so neither the per-term products nor their concatenation ever reach global memory.  s3 is the
// dominant contraction (2 kRows b1 b2 r_k3 flops per term); each thread owns an 8 x 8 register tile
// of it (rows (a1, x) = (tm, 0..3) and (32 + tm, 0..3), columns a2 = 4 tn + 0..3 and 32 + 4 tn + 0..3).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bf16.cuh"
#include "kernels.h"

namespace tks {

namespace {

constexpr int kRows = kProj3Rows;    // mode-1 rows per CTA
constexpr int kPad = 64;             // b2, b3 padded to 64
constexpr int kChunk = 16;           // mode-3 indices per chunk (at most)
constexpr int kGBytes = 16384;       // bytes of the core slice per chunk (at most)
constexpr int kGBuf = kGBytes + 32;  // + room for the 16-byte realignment of the slice
constexpr int kM = kRows * kPad;     // rows (a2, x) of the register block
constexpr int kThreads = 256;
constexpr int kR = TKS_MAX_RANK;

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

// Shared-memory layout (floats unless noted); the per-term operands A1, A2 are double-buffered by
// term parity, the per-chunk operands G, A3 by chunk parity.
struct Smem {
  float A1[2][kR * kRows];          // [i0][x]
  float A2[2][kR * kPad];           // [i1][a1]
  float A3[2][kChunk * kPad];       // [i2c][a2]
  float W1[kChunk * kR * kRows];    // [i2c][i1][x]
  float W2[kChunk * kM];            // [i2c][a1][x]
  __align__(16) unsigned char G[2][kGBuf];   // core slice G[:, :, c0 : c0 + nc], realigned to 16 bytes
};

// Chunks of a term: r2 split into ceil(r2 / cmax) nearly equal pieces.
template <typename CoreT>
__device__ __forceinline__ int chunk_max(const Proj3Term& T) {
  return min(kChunk, (int)(kGBytes / sizeof(CoreT)) / (T.r[0] * T.r[1]));
}

__device__ __forceinline__ float core_value(uint16_t h) { return bf16_float(h); }
__device__ __forceinline__ float core_value(float v) { return v; }

struct Pos {
  int k, c, nchunks;   // term, chunk of the term, chunks of the term
};

__device__ __forceinline__ void chunk_range(const Proj3Term& T, const Pos& p, int& c0, int& nc) {
  const int r2 = T.r[2];
  c0 = (p.c * r2) / p.nchunks;
  nc = ((p.c + 1) * r2) / p.nchunks - c0;
}

// Issue the asynchronous copies of one chunk (and, on its first chunk, of the term's A1 and A2)
// into buffer `buf`; returns the element shift of the core slice inside its buffer.
// Walks the elements e = tid, tid + kThreads, ... of a column-major (rows x cols) block as
// (row, col) = (e % rows, e / rows) without a division per element.
struct Walk {
  int row, col, drow, dcol;
  __device__ __forceinline__ Walk(int e, int rows)
      : row(e % rows), col(e / rows), drow(kThreads % rows), dcol(kThreads / rows) {}
  __device__ __forceinline__ void next(int rows) {
    row += drow;
    col += dcol;
    if (row >= rows) {
      row -= rows;
      col += 1;
    }
  }
};

// The job's fields as registers.
struct JobRegs {
  const float* AT[3];
  int64_t R[3];
  int64_t hs1, hs2;
  int b[3];
  int x0, rows;
};

template <typename CoreT>
__device__ __forceinline__ int issue_chunk(Smem& S, const JobRegs& J, const Proj3Term& T, const Pos& p, int buf,
                                           const Bases& bases) {
  const int tid = threadIdx.x;
  const int r0 = T.r[0], r1 = T.r[1];
  int c0, nc;
  chunk_range(T, p, c0, nc);
  if (p.c == 0) {
    const float* AT0 = J.AT[0] + T.roff[0];
    const float* AT1 = J.AT[1] + T.roff[1];
    float* A1 = S.A1[p.k & 1];
    float* A2 = S.A2[p.k & 1];
    for (Walk w(tid, r0); w.col < J.rows; w.next(r0))
      cp_async4(A1 + w.row * kRows + w.col, AT0 + w.row + J.R[0] * (J.x0 + w.col));
    for (Walk w(tid, r1); w.col < J.b[1]; w.next(r1))
      cp_async4(A2 + w.row * kPad + w.col, AT1 + w.row + J.R[1] * w.col);
  }
  const float* AT2 = J.AT[2] + T.roff[2] + c0;
  float* A3 = S.A3[buf];
  for (Walk w(tid, nc); w.col < J.b[2]; w.next(nc))
    cp_async4(A3 + w.row * kPad + w.col, AT2 + w.row + J.R[2] * w.col);
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

template <typename CoreT>
__device__ __forceinline__ bool advance(const Proj3Term* terms, int nterms, Pos& p) {
  if (++p.c < p.nchunks) return true;
  p.c = 0;
  if (++p.k >= nterms) return false;
  p.nchunks = (terms[p.k].r[2] + chunk_max<CoreT>(terms[p.k]) - 1) / chunk_max<CoreT>(terms[p.k]);
  return true;
}

template <typename CoreT>
__global__ void __launch_bounds__(kThreads, 2) project3_kernel(const Proj3Job* __restrict__ jobs, int njobs,
                                                                Bases bases) {
  extern __shared__ __align__(16) unsigned char p3raw[];
  Smem& S = *reinterpret_cast<Smem*>(p3raw);
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
  const int tid = threadIdx.x;
  const int tm = tid & 31, tn = tid >> 5;

  float acc[2][kRows][2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int x = 0; x < kRows; ++x)
#pragma unroll
      for (int nh = 0; nh < 2; ++nh)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[h][x][nh][j] = 0.f;

  // rows x >= J.rows of A1 stay zero (never copied into), so their accumulators stay zero
  for (int e = tid; e < 2 * kR * kRows; e += kThreads) (&S.A1[0][0])[e] = 0.f;
  __syncthreads();   // the zero fill lands before any copy into A1

  if (nterms > 0) {
    Pos cur{0, 0, (terms[0].r[2] + chunk_max<CoreT>(terms[0]) - 1) / chunk_max<CoreT>(terms[0])};
    int shift = issue_chunk<CoreT>(S, J, terms[0], cur, 0, bases);
    int buf = 0;
    bool more = true;
    while (more) {
      const Proj3Term& T = terms[cur.k];
      const int r0 = T.r[0], r1 = T.r[1];
      int c0, nc;
      chunk_range(T, cur, c0, nc);
      cp_async_wait_all();
      __syncthreads();   // this chunk is in shared memory; every thread is done with the other buffers
      Pos nxt = cur;
      more = advance<CoreT>(terms, nterms, nxt);
      int next_shift = 0;
      if (more) next_shift = issue_chunk<CoreT>(S, J, terms[nxt.k], nxt, buf ^ 1, bases);
      const float alpha = T.alpha;
      const float* A1 = S.A1[cur.k & 1];
      const float* A2 = S.A2[cur.k & 1];
      const float* A3 = S.A3[buf];
      const CoreT* Gs = reinterpret_cast<const CoreT*>(S.G[buf]) + shift;
      // s1: pair p = i1 + r1 i2c reads the contiguous core column G[:, i1, c0 + i2c]
      for (int p = tid; p < nc * r1; p += kThreads) {
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
        *reinterpret_cast<float4*>(S.W1 + kRows * p) =
            make_float4(alpha * w.x, alpha * w.y, alpha * w.z, alpha * w.w);
      }
      __syncthreads();
      // s2: a thread owns a1 = a1b .. a1b + 3 and x = 0..3 of one i2c
      {
        const int a1b = (tid & 15) * 4, i2c = tid >> 4;
        if (i2c < nc) {
          float w2[4][kRows];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int x = 0; x < kRows; ++x) w2[j][x] = 0.f;
          const float* w1 = S.W1 + kRows * (i2c * r1);
          for (int i1 = 0; i1 < r1; ++i1) {
            const float4 a = *reinterpret_cast<const float4*>(A2 + i1 * kPad + a1b);
            const float4 w = *reinterpret_cast<const float4*>(w1 + kRows * i1);
            const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              w2[j][0] = fmaf(av[j], w.x, w2[j][0]);
              w2[j][1] = fmaf(av[j], w.y, w2[j][1]);
              w2[j][2] = fmaf(av[j], w.z, w2[j][2]);
              w2[j][3] = fmaf(av[j], w.w, w2[j][3]);
            }
          }
          float* dst = S.W2 + i2c * kM + a1b * kRows;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            *reinterpret_cast<float4*>(dst + kRows * j) = make_float4(w2[j][0], w2[j][1], w2[j][2], w2[j][3]);
        }
      }
      __syncthreads();
      // s3: rank-nc update of the register block
      for (int i2c = 0; i2c < nc; ++i2c) {
        const float4 wlo = *reinterpret_cast<const float4*>(S.W2 + i2c * kM + tm * kRows);
        const float4 whi = *reinterpret_cast<const float4*>(S.W2 + i2c * kM + (32 + tm) * kRows);
        const float4 alo = *reinterpret_cast<const float4*>(A3 + i2c * kPad + tn * 4);
        const float4 ahi = *reinterpret_cast<const float4*>(A3 + i2c * kPad + 32 + tn * 4);
        const float wv[2][4] = {{wlo.x, wlo.y, wlo.z, wlo.w}, {whi.x, whi.y, whi.z, whi.w}};
        const float av[2][4] = {{alo.x, alo.y, alo.z, alo.w}, {ahi.x, ahi.y, ahi.z, ahi.w}};
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int x = 0; x < kRows; ++x)
#pragma unroll
            for (int nh = 0; nh < 2; ++nh)
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[h][x][nh][j] = fmaf(wv[h][x], av[nh][j], acc[h][x][nh][j]);
      }
      cur = nxt;
      shift = next_shift;
      buf ^= 1;
    }
  }

  // H (float64, mode-1 fastest): a lane writes the kRows consecutive rows of one (a1, a2); rows,
  // columns beyond b2, b3 hold whatever the uncopied padding of A2, A3 produced and are not written
  const int b0 = J.b[0], b1 = J.b[1], b2 = J.b[2];
  double* H = Hout;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int a1 = 32 * h + tm;
    if (a1 >= b1) continue;
#pragma unroll
    for (int nh = 0; nh < 2; ++nh)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int a2 = 32 * nh + 4 * tn + j;
        if (a2 >= b2) continue;
        double* dst = H + J.x0 + J.hs1 * a1 + J.hs2 * a2;
#pragma unroll
        for (int x = 0; x < kRows; ++x)
          if (x < J.rows) dst[x] = (double)acc[h][x][nh][j];
      }
  }
}

constexpr size_t kSmemBytes = sizeof(Smem);

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

void launch_proj3(const Proj3Job* jobs, int njobs, bool f32_cores, const Bases& bases, cudaStream_t stream) {
  if (f32_cores)
    project3_kernel<float><<<njobs, kThreads, kSmemBytes, stream>>>(jobs, njobs, bases);
  else
    project3_kernel<uint16_t><<<njobs, kThreads, kSmemBytes, stream>>>(jobs, njobs, bases);
}

}  // namespace tks

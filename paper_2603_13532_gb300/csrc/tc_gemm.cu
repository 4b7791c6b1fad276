// Grouped tensor-core GEMM for the contractions of the mixed-precision path on sm_103a.
//
// One CTA computes one 128 x BN output tile of one job.  Warp 0 (one elected thread) streams
// the bf16 planes of A and B through a ring of shared-memory stages with TMA (128-byte swizzle);
// warp 1 allocates acc TMEM accumulators (4 or 8) and (one elected thread) issues tcgen05.mma for
// every selected plane pair, 16 deep in k per instruction, k-block kb into accumulator kb % accj
// (accj: 4 for a job of K <= 1024, else 8, whatever the launch allocated),
// releasing each stage with tcgen05.commit; warps 2-5 read the accumulators back with
// tcgen05.ld (one TMEM lane quadrant each), add them and write the requested outputs.
// Every wait is bounded: on a timeout the kernel records TKS_ETIMEOUT,
// drains its own copies and MMAs (again bounded), frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bf16.cuh"
#include "kernels.h"
#include "tc.cuh"
#include "tc_shape.h"

namespace tks {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;                       // bf16 elements = 128 bytes = one swizzle row
constexpr int kATile = kBM * kBK * 2;         // 16 KB
static_assert(kBM == kTcBM && kBK == kTcBK, "the launch shape's tile sizes are the kernel's");
// Partial accumulators in TMEM: k-block kb goes to accumulator kb % accj and the epilogue adds
// them, so each float32 accumulator takes 1/accj of the K-steps (the rounding error of a long
// contraction whose products share a sign grows with the number of steps).  A job of K <= 1024
// takes four (at most four k-blocks each), a longer one eight.  tc_gemm_shape picks what a CTA
// allocates: four (256 TMEM columns, two CTAs per SM, one's loads and epilogue overlapping the
// other's products) when every job of the launch is short, else eight (all 512, one CTA per SM).

__device__ __forceinline__ void record_status_tc(Status* st, int code) {
  if (st) atomicCAS(&st->code, 0, code);
}

template <int BN>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const TcJob* __restrict__ jobs, int njobs, const CUtensorMap* __restrict__ maps, Bases bases,
                   Status* status, int stages, int na_max, int nb_max, int acc, long long kWaitCycles,
                   const volatile int* stall_word) {
  constexpr int kBTile = BN * kBK * 2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int stage_bytes = na_max * kATile + nb_max * kBTile;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)stages * stage_bytes);
  uint64_t* empty = full + stages;
  uint64_t* tmem_full = empty + stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tmem_full + 1);
  volatile int* err = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int lo = tile_job(jobs, njobs, (int)blockIdx.x);
  const TcJob& J = jobs[lo];
  const int local = blockIdx.x - J.tile_begin;
  const int tn = local % J.tiles_n, tm = local / J.tiles_n;
  const int m0 = tm * kBM, n0 = tn * BN;
  const int nk = (J.K + kBK - 1) / kBK;
  // the job's own partial accumulators: four for K <= kTcShortK, eight above (the launch allocates
  // acc = 8 whenever one of its jobs is longer), so that a job rounds the same whatever launch it
  // shares: one lane or several, one CTA per SM or two
  const int accj = J.K <= kTcShortK ? kTcAccShort : acc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(tmem_full, 1);
    *err = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, BN * acc);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  auto a_tile = [&](int s, int i) { return smem + (size_t)s * stage_bytes + (size_t)i * kATile; };
  auto b_tile = [&](int s, int j) {
    return smem + (size_t)s * stage_bytes + (size_t)na_max * kATile + (size_t)j * kBTile;
  };

  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < J.na; ++i) tc::prefetch_tmap(&maps[J.mapA[i]]);
      for (int j = 0; j < J.nb; ++j) tc::prefetch_tmap(&maps[J.mapB[j]]);
      int issued = 0;
      const uint32_t bytes = (uint32_t)(J.na * kATile + J.nb * kBTile);
      if (stall_word) {
        // failure-path test: wait for a word that nothing sets, so that this wait and the MMA
        // thread's run out and the kernel takes its timeout exit
        const long long t0 = clock64();
        while (*stall_word == 0) {
          if (clock64() - t0 > kWaitCycles) {
            *err = 1;
            break;
          }
          __nanosleep(256);
        }
      }
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % stages, round = kb / stages;
        if (*err || !tc::mbar_wait(&empty[s], (round & 1) ^ 1, kWaitCycles)) {
          *err = 1;
          break;
        }
        tc::mbar_expect_tx(&full[s], bytes);
        for (int i = 0; i < J.na; ++i) {
          if (J.a_mn) {
            // A stored with its row index fastest (e.g. Ucat itself): two 64-row boxes per plane
            tc::tma_load_2d(a_tile(s, i), &maps[J.mapA[i]], &full[s], m0, kb * kBK);
            tc::tma_load_2d(a_tile(s, i) + kATile / 2, &maps[J.mapA[i]], &full[s], m0 + kBM / 2, kb * kBK);
          } else {
            tc::tma_load_2d(a_tile(s, i), &maps[J.mapA[i]], &full[s], kb * kBK, m0);
          }
        }
        for (int j = 0; j < J.nb; ++j) tc::tma_load_2d(b_tile(s, j), &maps[J.mapB[j]], &full[s], kb * kBK, n0);
        issued = kb + 1;
      }
      // drain: every copy this thread issued has landed before the CTA tears down
      for (int kb = (issued > stages ? issued - stages : 0); kb < issued; ++kb)
        if (!tc::mbar_wait(&full[kb % stages], (kb / stages) & 1, kWaitCycles)) *err = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // an MN-major A (a_mn): two 64-row boxes 8 KB apart (LBO), 8-row k groups 1024 bytes apart
      // (SBO); a 16-deep k step moves its start by 2048 bytes (address field + 128), a K-major
      // tile's by 32 bytes (+ 2)
      const uint32_t idesc = J.a_mn ? tc::idesc_bf16_f32_amn(kBM, BN) : tc::idesc_bf16_f32(kBM, BN);
      const uint64_t astep = J.a_mn ? 128u : 2u;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % stages, round = kb / stages;
        if (*err || !tc::mbar_wait(&full[s], round & 1, kWaitCycles)) {
          *err = 1;
          break;
        }
        tc::fence_after_sync();
        // k-block kb accumulates into accumulator kb % accj; its first block starts it at zero
        const uint32_t d = tmem + (uint32_t)((kb % accj) * BN);
        uint32_t accum = kb >= accj ? 1u : 0u;
        for (int p = 0; p < J.npairs; ++p) {
          const uint32_t a0 = tc::smem_u32(a_tile(s, J.pa[p]));
          const uint32_t b0 = tc::smem_u32(b_tile(s, J.pb[p]));
          const uint64_t da = J.a_mn ? tc::sw128_mnmajor_desc(a0, kATile / 2, 1024) : tc::sw128_kmajor_desc(a0);
          const uint64_t db = tc::sw128_kmajor_desc(b0);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            tc::mma_bf16(d, da + astep * k, db + 2 * k, idesc, accum);
            accum = 1;
          }
        }
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(tmem_full);
      if (!tc::mbar_wait(tmem_full, 0, kWaitCycles)) *err = 1;
    }
  } else {
    // epilogue warps 2..5: TMEM lane quadrant q = warp % 4 holds rows 32q .. 32q+31
    bool ok = tc::mbar_wait(tmem_full, 0, kWaitCycles);
    ok = __all_sync(0xffffffffu, ok) && !*err;
    tc::fence_after_sync();
    if (ok) {
      const int q = warp & 3;
      const int row = m0 + 32 * q + lane;
      const TcEpi& E = J.epi;
      float* o32 = E.has_f32 ? at<float>(bases, E.f32) : nullptr;
      double* o64 = E.has_f64 ? at<double>(bases, E.f64) : nullptr;
      uint16_t* ob0 = E.nbf > 0 ? at<uint16_t>(bases, E.bf[0]) : nullptr;
      uint16_t* ob1 = E.nbf > 1 ? at<uint16_t>(bases, E.bf[1]) : nullptr;
      uint16_t* ob2 = E.nbf > 2 ? at<uint16_t>(bases, E.bf[2]) : nullptr;
      const int nacc = nk < accj ? nk : accj;
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 32) {
        // the partial accumulators of this column chunk (accj - 1 float32 additions: negligible
        // next to the K / (16 accj) roundings inside each accumulator; float64 arithmetic here
        // would run at the FP64 rate)
        float sum[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) sum[j] = 0.f;
        for (int a = 0; a < nacc; ++a) {
          uint32_t r[32];
          tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * BN + c0), r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 32; ++j) sum[j] += __uint_as_float(r[j]);
        }
        if (row < J.M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            if (col >= J.N) continue;
            const float v = E.alpha * sum[j];
            if (o32) o32[row * E.f32_m + col * E.f32_n] = v;
            if (o64) o64[row * E.f64_m + col * E.f64_n] = f32_to_f64_exact(v);
            if (ob0) {
              const int64_t off = row * E.bf_m + col * E.bf_n;
              const uint16_t h0 = bf16_bits(v);
              const float r1 = v - bf16_float(h0);
              ob0[off] = h0;
              if (ob1) {
                const uint16_t h1 = bf16_bits(r1);
                ob1[off] = h1;
                if (ob2) ob2[off] = bf16_bits(r1 - bf16_float(h1));
              }
            }
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, BN * acc);
  if (threadIdx.x == 0 && *err) record_status_tc(status, TKS_ETIMEOUT);
}

}  // namespace

cudaError_t prepare_tc_gemm() {
  return cudaFuncSetAttribute(tc_gemm_kernel<kTcBN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

void launch_tc_gemm(const TcJob* jobs, int njobs, int total_tiles, const void* maps, int na_max, int nb_max,
                    const Bases& bases, Status* status, long long wait_cycles, const int* stall_word,
                    int max_stages, int kmax, bool allow_two, cudaStream_t stream) {
  const TcShape sh = tc_gemm_shape(kmax, total_tiles, na_max, nb_max, max_stages, allow_two);
  tc_gemm_kernel<kTcBN><<<total_tiles, 192, sh.smem, stream>>>(jobs, njobs, static_cast<const CUtensorMap*>(maps),
                                                               bases, status, sh.stages, na_max, nb_max, sh.acc,
                                                               wait_cycles, stall_word);
}

}  // namespace tks

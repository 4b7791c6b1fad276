// Launch shape of the grouped tensor-core GEMM (tc_gemm_kernel): the shared-memory ring's stages,
// the dynamic shared memory, the number of 64-column TMEM partial accumulators and whether two CTAs
// share an SM.  Plain host arithmetic, included by the launch and compiled on its own by the CPU
// test that checks it against the SM's limits (228 KB of shared memory with 1 KB reserved per CTA,
// 512 TMEM columns).
#pragma once

#include <stddef.h>

namespace tks {

constexpr int kTcBM = 128;                     // output rows of a tile
constexpr int kTcBN = 64;                      // output columns of a tile (one accumulator)
constexpr int kTcBK = 64;                      // k-block: 64 bf16 = 128 bytes = one swizzle row
constexpr int kTcAccLong = 8;                  // accumulators of a CTA that has the SM to itself
constexpr int kTcAccShort = 4;                 // accumulators of each of two CTAs on an SM
constexpr int kTcShortK = 16 * kTcBK;          // longest K that two CTAs per SM take
constexpr int kTcTwoTiles = 32 * 152;          // most tiles a launch of K > 4 k-blocks takes on two
constexpr size_t kTcHalfSmem = 112 * 1024;     // ring budget of one of two CTAs
constexpr size_t kTcTwoFloor = 77 * 1024;      // above a third of the SM: no third CTA joins
constexpr size_t kTcOneFloor = 116 * 1024;     // above half the SM: the CTA owns all 512 columns
constexpr size_t kTcOneBudget = 220 * 1024;    // ring budget of a CTA alone on its SM

// 1 KB for aligning the ring to the 128-byte swizzle's 1024-byte pattern, the stages (na A planes
// of 128 x 64 and nb B planes of bn x 64 bf16 each), 2 stages + 1 mbarriers and the TMEM slot.
inline size_t tc_gemm_smem_bytes(int stages, int na_max, int nb_max, int bn) {
  return 1024 + (size_t)stages * ((size_t)na_max * kTcBM * kTcBK * 2 + (size_t)nb_max * bn * kTcBK * 2) +
         8 * (2 * (size_t)stages + 1) + 16;
}

// Deepest ring (4 down to 2 stages, else 1) within `budget` bytes.
inline int tc_gemm_ring(int na_max, int nb_max, int bn, size_t budget) {
  for (int s = 4; s >= 2; --s)
    if (tc_gemm_smem_bytes(s, na_max, nb_max, bn) <= budget) return s;
  return 1;
}

struct TcShape {
  bool two;      // two CTAs per SM, each with kTcAccShort accumulators; else one with kTcAccLong
  int stages;    // ring stages
  size_t smem;   // dynamic shared memory of a CTA, bytes
  int acc;       // 64-column TMEM accumulators a CTA allocates; k-block kb goes to kb % acc
};

// kmax: the launch's longest contraction; total_tiles: its 128 x 64 output tiles; na_max, nb_max:
// the most bf16 planes of an A or B operand; max_stages: a cap on the ring (0 = none); allow_two:
// false when the launch runs beside other streams' kernels that may hold all of an SM's TMEM
// columns (two CTAs of 77-113 KB could share an SM with one of them and wait for columns).
//
// Two CTAs per SM for short contractions (K <= kTcShortK) of at most kTcTwoTiles tiles (a few
// tiles an SM, whose TMA set-up, products and epilogue one CTA per SM would run in turn) and for
// those of at most four k-blocks (epilogue-heavy).  Short contractions of more tiles keep one CTA
// per SM (measured no faster on two).  The shape changes no result: a job of K <= kTcShortK always
// spreads its k-blocks over four accumulators and a longer one over eight (the kernel's per-job
// count), so only what a CTA allocates differs.
inline TcShape tc_gemm_shape(int kmax, int total_tiles, int na_max, int nb_max, int max_stages,
                             bool allow_two = true) {
  TcShape sh;
  sh.two = allow_two && kmax <= kTcShortK && (total_tiles <= kTcTwoTiles || kmax <= kTcAccShort * kTcBK);
  sh.stages = tc_gemm_ring(na_max, nb_max, kTcBN, sh.two ? kTcHalfSmem : kTcOneBudget);
  if (max_stages > 0 && sh.stages > max_stages) sh.stages = max_stages;
  const size_t need = tc_gemm_smem_bytes(sh.stages, na_max, nb_max, kTcBN);
  const size_t floor = sh.two ? kTcTwoFloor : kTcOneFloor;
  sh.smem = need > floor ? need : floor;
  sh.acc = sh.two ? kTcAccShort : kTcAccLong;
  return sh;
}

}  // namespace tks

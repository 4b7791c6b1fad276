// Internal descriptor tables shared by the host planner and the kernels.
//
// Every operand in a launch table is (base id, byte offset).  Base ids name the
// buffers an execute call binds: the workspace, the caller's output buffers and
// "absolute" (the offset is a device address remembered at plan time, used for
// the caller's input cores and factors).  Binding at launch time lets one plan
// serve every entry point without copying tables again.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "tks.h"

namespace tks {

constexpr int MAXD = TKS_MAX_ORDER;

enum BaseId : int32_t {
  B_NONE = -2,   // no operand
  B_ABS = -1,    // offset is an absolute device address
  B_WS = 0,      // workspace
  B_OMEGA = 1,   // Omega buffer (caller's for tks_generate_omega, else workspace)
  B_Y = 2,       // sketch buffer
  B_Q = 3,       // basis buffer
  B_H = 4,       // projected core buffer
  B_OUT = 5,     // recompression output (cores and factors)
  B_RANKS = 6,   // recompression output ranks (int32)
  B_HBAR = 7,    // backward: dL/dH
  B_DCORE = 8,   // backward: core gradients
  B_DFAC = 9,    // backward: factor gradients
  B_EVALS = 10,  // effective subrank: eigenvalues of the weighted Gram matrices
  B_SRANK = 11,  // effective subrank: ranks (int32)
  B_ELL = 12,    // effective subrank: ell = rank + oversampling (int32)
  NBASE = 13
};

struct Bases {
  char* p[NBASE];
};

struct Operand {
  int32_t base;
  int32_t pad;
  int64_t off;   // bytes
};

template <typename T>
__host__ __device__ inline T* at(const Bases& b, const Operand& o) {
  return reinterpret_cast<T*>(o.base < 0 ? reinterpret_cast<char*>(o.off) : b.p[o.base] + o.off);
}

// ---------------------------------------------------------------------------
// Generic strided float64 GEMM job: C[i,j] = alpha * sum_k A[i,k] B[k,j] (+ beta C).
// The reduction index k splits into k0 = k % K1, k1 = k / K1 with separate strides so
// that an unfolding whose columns are a two-level index (e.g. the Gram matrix of a
// mode-n unfolding) is a single job.  batch repeats the job with extra strides.
// With ksplit > 1 each K chunk writes partial sums to P (ksplit x batch x M x N,
// column-major) and a second kernel adds the chunks in order, so the result does
// not depend on scheduling.
struct GemmJob {
  int32_t M, N, K, K1;
  int32_t batch, ksplit, kchunk;
  int32_t tiles_m, tiles_n;
  int32_t tile_begin;
  int64_t red_begin;            // prefix over split jobs of batch * M * N (reduction kernel)
  Operand A, B, C, P;
  int64_t a_m, a_k0, a_k1, a_b;
  int64_t b_n, b_k0, b_k1, b_b;
  int64_t c_m, c_n, c_b;
  double alpha, beta;
};

// Gaussian draws of one (problem, mode): Omega (n x s, column-major).
struct OmegaJob {
  Operand out;
  Operand plane;       // bf16 copy (same layout) when has_plane
  int64_t count;       // n * s
  int64_t begin;       // prefix over jobs (elements)
  int32_t problem, mode;
  int32_t bf16;        // float32 draws (gaussian4_f32) rounded to bfloat16
  int32_t has_plane;
};

// Element types of typed operands.
enum ElemType : int32_t { T_F64 = 0, T_F32 = 1, T_BF16 = 2 };

// Float32 CUDA-core GEMM job with typed operands (same index scheme as GemmJob):
//   C[i,j] = alpha * sum_k A[i,k] B[k,j], written as float32, float64 and/or split into
//   bfloat16 planes (hi, mid, lo), all at C + i c_m + j c_n + batch c_b.
struct SimtJob {
  int32_t M, N, K, K1;
  int32_t batch, tiles_m, tiles_n, tile_begin;
  Operand A, B;
  int32_t a_type, b_type;
  int64_t a_m, a_k0, a_k1, a_b;
  int64_t b_n, b_k0, b_k1, b_b;
  Operand c32, c64, cb[3];
  int32_t has_c32, has_c64, nbf, pad;
  int64_t c_m, c_n, c_b;
  float alpha, pad2;
};

// Khatri-Rao / Kronecker core sketch in float32: G_k (bf16) and M_j (float32) in, V_kn out as
// bfloat16 planes of Vcat_n (element (r, c) at r + ldv c).
struct CoreSketchF32Job {
  Operand core;
  Operand M[MAXD];
  Operand V[3];
  int32_t d, n, kron, ldv;
  int32_t r[MAXD];
  int32_t roff[MAXD];
  int32_t R[MAXD];
  int32_t s[MAXD];
  int32_t S, pad;
  float alpha, pad2;
  int64_t count;
  int64_t begin;
};

// Mode product with a small matrix (ST-HOSVD truncation and final factors):
// Y[l + L (c + rmax r)] = sum_a X[l + L (a + b r)] P[a + b c] for l < L, r < Rr, c < rmax.
// float32 kernel: X typed (T_F64 / T_F32), P float32, Y typed, rmax <= 64; float64 kernel: X, P
// and Y float64.
struct TtmJob {
  Operand X, P, Y;
  int32_t x_type, y_type;
  int64_t L, Rr;
  int32_t b, rmax;
  int32_t tile_begin, tiles;
};

// Khatri-Rao core sketches of all three modes of one order-3 term (stage b, float32), one CTA per
// term; requires s <= 64 and ranks <= kSketch3MaxRank.
constexpr int kSketch3MaxRank = 32;

struct Sketch3Job {
  Operand core;          // bf16 core, mode-1 fastest
  Operand M[3];          // float32 M_m = Ucat_m^T Omega_m: element (i, c) at i + R_m c
  Operand V[3][3];       // bf16 planes of Vcat_n: element (i, c) at i + ldv_n c
  int32_t r[3], roff[3], R[3], ldv[3];
  int32_t s;
  float alpha;
  int32_t pad[2];
};

// Khatri-Rao core sketches of all four modes of one order-4 term (stage b, float32), one CTA per
// term; requires s <= 64 and ranks <= kSketch4MaxRank.  The core is staged in slices of kc mode-1
// indices.
constexpr int kSketch4MaxRank = 24;

struct Sketch4Job {
  Operand core;          // bf16 core, mode-1 fastest
  Operand M[4];          // float32 M_m = Ucat_m^T Omega_m: element (i, c) at i + R_m c
  Operand V[4][3];       // bf16 planes of Vcat_n: element (i, c) at i + ldv_n c
  int32_t r[4], roff[4], R[4], ldv[4];
  int32_t s, kc;
  float alpha;
  int32_t pad;
};

// Fused order-3 projection (stage c; float32 on the CUDA cores, split bf16 on the tensor cores):
// one CTA per (problem, kProj3Rows mode-1 rows of H), requires b_2, b_3 <= 64.  The job table is
// followed by the Proj3Term records of all problems; job j reads terms [term_begin, term_begin +
// nterms) of that array.  A chunk stages at most kProj3SliceBytes of a core, and at least one
// mode-3 slice G[:, :, i3] must fit.
constexpr int kProj3Rows = 4;
constexpr int kProj3SliceBytes = 12288;
constexpr int kProj3Chunk = 16;        // mode-3 indices of a chunk (at most): K of one MMA
constexpr int kProj3W1Floats = 2048;   // first-stage products of a chunk (at most)

// Mode-3 indices per chunk of a term with ranks r and core elements of `elem` bytes: the chunk's
// core slice fits kProj3SliceBytes and its first-stage products kProj3W1Floats (odd row stride).
inline int proj3_chunk(const int32_t r[3], int elem) {
  int c = kProj3Chunk;
  c = std::min(c, kProj3SliceBytes / elem / (r[0] * r[1]));
  c = std::min(c, kProj3W1Floats / (kProj3Rows * (r[1] | 1)));
  return c;
}

struct Proj3Term {
  Operand core;          // bf16 core of the term, mode-1 fastest
  int32_t r[3];          // term ranks
  int32_t roff[3];       // first row of the term in A_n^T
  float alpha;           // term weight
  int32_t chunk;         // mode-3 indices per chunk: chunk c covers [c chunk, min(r3, (c + 1) chunk))
};

struct Proj3Job {
  Operand AT[3];         // float32 A_n^T = (Q_n^T Ucat_n)^T: element (i, a) at i + R_n a
  Operand H;             // float64 H, element (a0, a1, a2) at a0 + hs1 a1 + hs2 a2
  int32_t R[3], b[3];
  int32_t x0, rows;      // mode-1 rows [x0, x0 + rows), rows <= kProj3Rows
  int32_t term_begin, nterms;
  int64_t hs1, hs2;      // strides of a1 and a2 in H (b0 and b0 b1 for an order-3 core)
  int32_t pad[2];
};
static_assert(sizeof(Proj3Job) % 16 == 0 && sizeof(Proj3Term) % 16 == 0, "term records follow the jobs");

// Order-4 problems on the fused projection: G'_k(a1) = alpha_k G_k x_2 A_2k[a1, :] (r0 x r2 x r3,
// float32) for every row a1 of A_2k, so that H[:, a1, :, :] is the order-3 projection of the
// G'_k(a1) with A_1k, A_3k, A_4k.  One CTA per (term, mode-4 index i3).
struct Fold4Job {
  Operand core;          // bf16 G_k, mode-1 fastest (r0, r1, r2, r3)
  Operand AT1;           // float32 A_2^T: element (i, a) at i + R1 a, term rows from roff1
  Operand out;           // float32; G'_k(a1)[i0, i2, i3] at out + a1 r0 r2 r3 + i0 + r0 (i2 + r2 i3)
  int32_t r[4];
  int64_t R1;
  int32_t roff1, b1;
  float alpha;
  int32_t i3;
};

// Order-3 chain of one term for rows [a0, a0 + AB) of mode 1 (stage c2, float32):
//   T[a0, a1, c] = alpha sum_{i0, i1} A1[a0, i0] A2[a1, i1] G[i0, i1, c]
// with A_t[a, i] = AT_t[(roff_t + i) + R_t a]; written as bf16 planes of Tcat at
// (roff_2 + c) + ldT (a0 + b0 a1).
struct Chain3Job {
  Operand core, AT[2], T[3];
  int32_t r[3], roff[3], R[2], b[2];
  int32_t a0, rows, ldT, pad;
  float alpha, pad2;
};

// Split a float64 matrix (rows x cols, element (i, j) at i + ld_src j) into bf16 planes
// hi + mid + lo (element (i, j) at i + ld_dst j).
// Split a float64 matrix into three bf16 planes; the launch covers each job in tiles of
// kSplitTile elements (column-major order), tiles [tile_begin, tile_begin + ceil(count / kSplitTile)).
constexpr int kSplitTile = 1024;
struct SplitJob {
  Operand src;
  Operand dst[3];
  int64_t rows, cols, ld_src, ld_dst;
  int64_t count, begin;
  int32_t trans;        // trans: element (i, j) goes to j + ld_dst i (else i + ld_dst j)
  int32_t tile_begin;
};

// Transpose a bf16 matrix: dst[j + ld_dst i] = src[i + ld_src j] (src rows x cols).
struct TransposeJob {
  Operand src, dst;
  int32_t rows, cols;
  int64_t ld_src, ld_dst;
  int32_t tiles_r, tiles_c, tile_begin, pad;
};

// Structured core sketch of one (term, mode n): V_kn (r_kn x S_n) into rows
// [roff_n, roff_n + r_kn) of Vcat_n (R_n x S_n, column-major).
struct CoreSketchJob {
  Operand core;                 // G_k, float64, mode 1 fastest
  Operand M[MAXD];              // M_j = Ucat_j^T Omega_j (R_j x s_j), float64
  Operand V;                    // Vcat_n
  int32_t d, n, kron;
  int32_t r[MAXD];
  int32_t roff[MAXD];
  int32_t R[MAXD];
  int32_t s[MAXD];              // Omega columns per mode
  int32_t S;                    // columns of V (s for KRP, prod_{j != n} s_j for Kron)
  int32_t Rn;                   // leading dimension of Vcat_n
  double alpha;
  int64_t count;                // r_kn * S
  int64_t begin;
};

// Householder QR of Y (n x S) giving Q (n x b), b = min(n, S), diag(R) >= 0.
struct QrJob {
  Operand Y, W, Q, tau;         // W: n x S work copy, tau: S doubles
  Operand gate;                 // when gate.base != B_NONE, the job runs only if the int32 there is
                                // nonzero (the CholeskyQR path asked for the Householder fallback)
  int32_t n, S, b, pad;
};

// Tensor-core GEMM (tcgen05, bf16 inputs, f32 accumulation in TMEM):
//   D (M x N) = alpha * sum_{p < npairs} A_{pa[p]} B_{pb[p]}^T
// A_i (M x K) and B_j (N x K) are bfloat16 planes in K-major layout read by TMA through the
// tensor maps mapA[i] / mapB[j]; rows beyond M or N and k beyond K read as zero.  A float32
// operand enters as up to three planes hi + mid + lo (each bfloat16, their sum equals the
// float32 value to about 2^-24 relative), and the pair list selects the products kept.
// The epilogue writes any of: float32 D, float64 D, and D split again into bf16 planes for
// the next contraction, each with its own (row, column) element strides.
struct TcEpi {
  Operand f32, f64, bf[3];
  int64_t f32_m, f32_n, f64_m, f64_n, bf_m, bf_n;
  int32_t has_f32, has_f64, nbf;
  float alpha;
};

struct TcJob {
  int32_t M, N, K;
  int32_t tiles_m, tiles_n, tile_begin;
  int32_t na, nb, npairs;
  int32_t a_mn;          // 1: the A maps have the row index innermost (box 64 rows x 64 k), read MN-major
  int32_t mapA[3], mapB[3];
  uint8_t pa[8], pb[8];
  TcEpi epi;
};

// Householder QR in float32 of a tall matrix A (rows x cols) read through a two-level row
// index: element (i, j) with i = i0 + L0 i1 at src[i0 s0 + i1 s1 + j sc] (src of type src_type).
// Outputs: the orthonormal factor Q (rows x b, float64, diag(R) >= 0) and/or the triangular
// factor R (b x b, float32, column-major), b = min(rows, cols).
struct QrF32Job {
  Operand src, W, tau, Q, R;
  Operand Qp[3];         // register kernel: Q also as bf16 planes hi/mid/lo (same layout) when nplanes
  int32_t src_type, want_q, want_r, b;
  int64_t rows, cols, L0, s0, s1, sc;
  int32_t nplanes, pad;
};

// One block of a TSQR level: rows [row_begin, row_begin + rows) x cols of a (typed, two-level
// row index) source are factored by Householder; the b x b triangular factor (rows below
// min(rows, cols) zero) is written at rows [dst_row0, dst_row0 + cols) of dst (column-major,
// leading dimension dst_ld; float32 for the float32 kernel, float64 with a float64 source for
// the float64 kernel).  Stacking the blocks' factors and
// factoring again gives the triangular factor of the whole matrix.
struct TsqrJob {
  Operand src, dst;
  Operand gate;          // float64 kernel: when gate.base != B_NONE, the block runs only if the int32
                         // there is nonzero (the CholeskyQR path asked for the Householder fallback)
  int32_t src_type, rows, cols;
  int32_t tri;           // float64 kernel: 0 = dense rows; k = the rows interleave k stacked upper
                         // triangular factors (row i = factor + k r), so column j is zero where r > j
  int64_t row_begin, L0, s0, s1, sc;
  int64_t dst_row0, dst_ld;
};

// One-sided (Hestenes) Jacobi SVD of the b x b factor R of H_(n)^T = Q~ R: its right singular
// vectors are the left singular vectors of H_(n).  Selects the rank (min(rmax, b), or the
// tolerance rule of Alg. 2 with theta = tol^2 ||H||^2 / d fixed at the first mode) and writes
// P = leading right singular vectors (b x rmax, zero-padded) and the b singular values sv, all
// float32 for the float32 kernel and float64 for the float64 kernel (theta is float64 in both).
struct SvdJob {
  Operand R, P, sv, theta, rank;
  Operand err;           // float64 [1 + TKS_MAX_ORDER]: ||H||^2 (first mode) and each mode's discarded
                         // squared singular values, at index 1 + mode (B_NONE: not recorded)
  int32_t b, rmax, first_mode, order, mode, pad;
  double tol;
};

// Relative truncation error of one problem's ST-HOSVD from the energies its SVD jobs recorded.
struct TruncErrJob {
  Operand err;           // float64 [1 + TKS_MAX_ORDER] as in SvdJob
  Operand out;           // float64: sqrt(sum of the discarded energies / ||H||^2)
  int32_t d, pad;
};

// Float64-accurate mode product on the tensor cores (the ST-HOSVD truncation of TKS_MIXED):
//   Y[l + L (c + rmax r)] = sum_a X[l + L (a + K r)] P[a + K c]
// by exact integer slices (the Ozaki scheme).  Each row of X (fibre q = l + L r) and of P^T (column c)
// is scaled by a power of two 2^e with |x| < 2^e over the row and cut into kOzSlices signed 7-bit
// digits, x = 2^e sum_s d_s 2^(-7 s) up to 2^(e - 56); the digits are bfloat16 integers, their
// products exact, and every sum over K <= TKS_MAX_BASIS of them an integer below 2^21, so the
// tensor cores accumulate each level s + t of digit pairs exactly in float32.
constexpr int kOzSlices = 8;     // 56 bits of every row
constexpr int kOzLevels = 8;     // digit pairs with s + t <= 9 (1-based): levels 2..9

// Cuts the rows of a float64 matrix into digit planes: row q (q < rows) holds element a (a < K) at
// src[l + L a + L K r] with q = l + L r; plane s of row q goes to planes at element
// (s * rows_pad + q) * ld + a, and the row's exponent e to expo[q].
struct OzSliceJob {
  Operand src, planes, expo;
  Operand kexp;          // int32 per K index a (B_NONE: none): row q is sliced as x[q][a] 2^kexp[a]
  int64_t rows, L, rows_pad;
  int32_t K, ld;
  int32_t tile_begin, tiles;
};

// One 128 x 64 output tile per CTA: A = digit planes of the X rows (TMA maps mapA[s]), B = digit
// planes of the P columns (mapB[s]); the kOzLevels accumulators live in TMEM.
struct OzGemmJob {
  int32_t M, N, K;
  int32_t tiles_m, tiles_n, tile_begin;
  int32_t mapA[kOzSlices], mapB[kOzSlices];
  Operand expA, expB;    // int32 row exponents of X and of P^T (expA.base == B_NONE: X's are all 0)
  Operand Y;             // float64: element (q, c) at Y[l + L (c + rmax r)], q = l + L r
  int64_t L;
  int32_t rmax;
  int32_t a_mn;          // 1: mapA[s] are column digit planes (box 64 rows x 64 k, row index fastest),
                         // read MN-major as two boxes per 128-row tile; 0: row planes, K-major
};

// Shifted CholeskyQR3 of X = H_(n)^T (P x b, element (i = l + L r, a) at src[l + L a + L b r]) with
// float64-accurate Gram matrices on the tensor cores (TKS_MIXED).  X is cut into digits against one
// exponent per COLUMN, e_a with |X[i][a]| < 2^e_a, in 64-row tiles (one CTA per tile, two launches):
//   oz_xmax:  the largest biased exponent field of each column over the tile -> part[tile][a];
//   oz_xdig:  e_a from the partials of the matrix's tiles (the first tile stores them at expo[a]),
//             then the digits: plane s of column a at colP + (s * 64 + a) * ldP (element i).  The
//             Gram reads these planes K-major (K = rows) and X Rinv reads them MN-major (K = columns);
//             with column exponents X Rinv needs no row exponents: the Cholesky step writes Rinv with
//             row a scaled by 2^e_a.
struct OzXSliceJob {
  Operand src, part, expo, colP;
  int64_t P, L, ldP, rows_pad;
  int32_t b, tiles, tile_begin, pad;
};

// G = X^T X (b x b, b <= 64) from the column digit planes (TMA maps map[s], box 64 k x 64 rows),
// one CTA per job, K = P in blocks of 64; G float64 at G[i + b j].
struct OzGramJob {
  int32_t map[kOzSlices];
  Operand expo, G;
  int64_t P;
  int32_t b, pad;
};

// One Cholesky step of shifted CholeskyQR3 (pass 1..3) on G (b x b, float64), one CTA per job:
// R = chol(G + shift I) (shift only in pass 1), Rinv = R^-1 for the next X <- X Rinv, Racc <- R Racc;
// the last pass writes Racc (the triangular factor of X) to Rout and clears *fallback, a pivot below
// the pass's bound sets *fallback (the Householder TSQR then factors X instead).
struct CholJob {
  Operand G, Rinv, Racc, Rout, fallback;
  Operand xexp;          // int32 column exponents of X: Rinv row a is written times 2^xexp[a] (B_NONE: none)
  int64_t P;
  int32_t b, pass;       // pass 1 starts Racc; later passes read *fallback
  int32_t shift, last;   // shift: add s I first (shifted CholeskyQR3); last: write Racc to Rout
  double pivot_tol;      // a pivot d_j <= pivot_tol G_jj (or not positive) sets *fallback
};

// Effective subrank heuristic (Alg. 5), float64 throughout.
//
// Term weight w_k = |alpha_k| ||G_k||_F, written as the weight of each of the term's columns of
// every Ucat_m (so the energy-weighted concatenation is V_m = Ucat_m diag(wcol_m)).
struct WeightJob {
  Operand core;           // typed (T_F64 / T_BF16), `count` elements
  Operand wcol[MAXD];     // float64: this term's r_km column weights in mode m
  int64_t count;
  int32_t type, d;
  int32_t r[MAXD];
  double alpha;
};

// Weighted Gram matrix of one (problem, mode) in float64, computed in 64 x 64 tiles of the lower
// triangle and mirrored:
//   aat = 0:  B = W Ucat^T Ucat W     (m = R, used when R <= n)
//   aat = 1:  B = Ucat W^2 Ucat^T     (m = n, used when n < R)
// with W = diag(wcol).  The two products have the same nonzero eigenvalues.
struct GramJob {
  Operand U, wcol, B;     // U typed, n x R column-major (ld n); B m x m (ld m)
  int64_t n;
  int32_t R, m, type, aat;
  int32_t tiles, tile_begin;   // T (T + 1) / 2 lower-triangle tiles, T = ceil(m / 64)
};

// Eigenvalues of one weighted Gram matrix and the rank rule of Alg. 5: Householder
// tridiagonalization of B (overwritten) into diagonal d and off-diagonal e, implicit QR steps
// on (d, e), then rank = min{r >= 1 : sum_{j > r} lambda_j <= eps^2 / order * sum_j lambda_j}
// over the eigenvalues clamped at zero, and ell = rank + p.
struct SubrankJob {
  Operand B, d, e, ev;    // ev: the m eigenvalues in descending order (float64)
  Operand rank, ell;      // int32 outputs
  int32_t m, order, p, pad;
  double eps;
  int32_t* steps;         // device: reduction steps the tridiagonalization executed (its early end)
};

struct Status {
  int32_t code;                 // first tks_status recorded by a kernel
  int32_t pad;
};

#ifdef __CUDACC__
// The job that owns tile t of a grouped launch (jobs in tile order, job j covering tiles
// [jobs[j].tile_begin, jobs[j + 1].tile_begin)).  A batch of equal problems gives every job the same
// tile count, so the guess from the first job's count is checked first: two rounds of loads from the
// job table instead of the log2(njobs) dependent rounds of a binary search, which remains the fallback.
template <class Job>
__device__ __forceinline__ int tile_job(const Job* __restrict__ jobs, int njobs, int t) {
  if (njobs <= 1) return 0;
  const int t0 = jobs[0].tile_begin, per = jobs[1].tile_begin - t0;
  if (per > 0) {
    const int j = (t - t0) / per;
    if (j >= 0 && j < njobs && jobs[j].tile_begin <= t && (j + 1 == njobs || jobs[j + 1].tile_begin > t)) return j;
  }
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}
#endif

// Sets the thread-local message returned by tks_last_error (host code of every entry point).
void set_last_error(const std::string& msg);

}  // namespace tks

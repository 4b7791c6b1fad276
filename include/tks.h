/*
 * tks.h -- C ABI of the GB300 (sm_103a) library for sketched recompression of
 * sums of Tucker tensors (R. Smith et al., "Efficient Sketching-Based Summation
 * of Tucker Tensors", arXiv 2603.13532).
 *
 * A problem is a sum of K Tucker terms X = sum_k alpha_k G_k x_1 U_k^(1) ... x_d U_k^(d)
 * (Eq. TuckerDecompositionModeProd; term weights as in TuckerAxby, Alg. 1).  The
 * library recompresses X without forming it (KronSum-Tucker, Alg. 3; KRPSum-Tucker,
 * Alg. 4):
 *   stage (a)  M_kj = U_k^(j)^T Omega_j with Gaussian Omega_j (Sec. 3.1, factor reuse)
 *   stage (b)  Y_n = sum_k U_k^(n) V_kn with the Khatri-Rao or Kronecker core sketch
 *              V_kn (Eqs. KRP_sketch_unfolding / Kron_sketch_unfolding), Q_n = qr(Y_n)
 *   stage (c)  H = sum_k G_k x_1 (Q_1^T U_k^(1)) ... x_d (Q_d^T U_k^(d)) (Sec. 3.3)
 *   final      ST-HOSVD truncation of H (Alg. 2 phase 2), U~_n = Q_n P_n.
 * Many independent problems of different sizes go into one plan and run in grouped
 * launches.
 *
 * Conventions for every entry point
 *   - Matrices are column-major.  Tensors are stored with mode 1 fastest, which is
 *     the unfolding order of Eq. unfolding_index.
 *   - "device" pointers are CUDA global-memory addresses on the plan's device, "host"
 *     pointers are ordinary CPU memory.  The caller owns every buffer it passes; the
 *     library allocates device memory only inside tks_plan_create (descriptor tables
 *     and a status word) and frees it in tks_plan_destroy.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Execute calls only
 *     enqueue work and return; results and the device status word are valid after the
 *     stream completes.  tks_sync_status synchronizes and reports device-side errors.
 *   - Errors are returned as tks_status (never exceptions); tks_last_error() gives a
 *     thread-local message for the last failing call on that thread.
 *   - Calls on the same plan must not run concurrently on different streams: they
 *     share the plan's status word (and the workspace, if the same one is passed).
 */
#ifndef TKS_H
#define TKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TKS_API __attribute__((visibility("default")))
#else
#define TKS_API
#endif

#define TKS_MAX_ORDER 6      /* tensor order d: 2 <= d <= TKS_MAX_ORDER */
#define TKS_MAX_RANK 64      /* per-term rank r_km: 1 <= r_km <= min(n_m, TKS_MAX_RANK) */
#define TKS_MAX_BASIS 96     /* columns of Q_n, b_n = min(n_n, S_n) <= TKS_MAX_BASIS */

typedef enum {
  TKS_OK = 0,
  TKS_EINVAL = 1,        /* invalid argument; nothing was enqueued */
  TKS_ENOMEM = 2,        /* a device allocation inside tks_plan_create failed */
  TKS_ECUDA = 3,         /* a CUDA runtime call failed (message in tks_last_error) */
  TKS_ETIMEOUT = 4,      /* a bounded device-side wait ran out (kernel returned early) */
  TKS_ENONFINITE = 5,    /* a NaN or Inf reached the sketch or the projected core */
  TKS_ENOCONV = 6,       /* a Jacobi SVD of the ST-HOSVD hit its sweep limit */
  TKS_EUNSUPPORTED = 7   /* valid input outside the limits the library supports */
} tks_status;

typedef enum { TKS_SKETCH_KRON = 0, TKS_SKETCH_KRP = 1 } tks_sketch;

typedef enum {
  TKS_FP64 = 0,   /* every stage in float64 on CUDA cores (the plain FP64 GPU path) */
  TKS_MIXED = 1,  /* contractions on tcgen05 tensor cores with bfloat16 operands (a float32
                     operand is split into bfloat16 planes) and float32 accumulation; QR and
                     ST-HOSVD as in TKS_FP64 */
  TKS_MIXED_F32LA = 2  /* contractions as TKS_MIXED; QR of Y_n and ST-HOSVD in float32 with
                          backward-stable algorithms (Householder QR, one-sided Jacobi SVD of
                          the triangular factor of H_(n)^T; no Gram matrices) */
} tks_precision;

typedef enum { TKS_DT_F64 = 0, TKS_DT_BF16 = 1 } tks_dtype;

/* One Tucker sum.  All arrays described as host are read during tks_plan_create only;
 * the device pointers are remembered by the plan and read by every execute call. */
typedef struct {
  int32_t order;                /* d */
  const int64_t* dims;          /* host [d]: n_1..n_d, each >= 1 */
  int32_t num_terms;            /* 1 <= K <= 2^20 */
  const int32_t* ranks;         /* host [K*d]: ranks[k*d + m] = r_km */
  const int32_t* target_ranks;  /* host [d]: target rank per mode, >= 1 */
  const int32_t* oversampling;  /* host [d]: oversampling p_n >= 0; ell_n = target_n + p_n <= 2^21 */
  const double* alpha;          /* host [K] term weights, or NULL for all ones */
  const void* cores;            /* device: the K cores packed back to back, term k's core
                                   (r_k1 x ... x r_kd, mode 1 fastest) starting at element
                                   sum_{k'<k} prod_m r_k'm; element type = params dtype */
  const void* const* factors;   /* host [d] of device pointers: factors[m] is the
                                   concatenated factor Ucat_m = [U_1^(m) ... U_K^(m)],
                                   n_m x R_m column-major (ld = n_m), R_m = sum_k r_km
                                   (the TuckerAxby layout, Alg. 1) */
} tks_problem;

typedef struct {
  tks_sketch sketch;            /* Kronecker (Alg. 3) or Khatri-Rao (Alg. 4) */
  tks_precision precision;      /* TKS_FP64 needs dtype F64; the mixed modes need dtype BF16
                                   and n_m % 8 == 0 with 16-byte aligned factors */
  tks_dtype dtype;              /* element type of cores and factors */
  uint64_t seed;                /* key of the Gaussian draws (Philox4x64-10) */
  double trunc_tol;             /* 0: keep min(target_n, b_n) columns per mode; > 0: the
                                   relative tolerance rule of Alg. 2, capped by the target */
  int32_t omega_lowprec;        /* 0: the precision's own Gaussian draws (float64 Box-Muller for
                                   TKS_FP64, float32 rounded to bfloat16 for the mixed modes);
                                   1: the mixed modes' draws for every precision, so that a
                                   TKS_FP64 plan computes with the Omega of a mixed plan (an
                                   arithmetic-only comparison of the two) */
  int32_t lanes;                /* 0 or 1: tucker_sum_recompress is one sequence of grouped launches.
                                   2..8 (mixed modes): the problems are split into that many
                                   contiguous groups whose launch sequences run on concurrent
                                   streams, forked from and joined back to the caller's stream (the
                                   latency-bound stages of one group overlap the others' work);
                                   results are identical.  Ignored by TKS_FP64 and by the other
                                   entry points. */
  /* Schedule knobs (0 = the built-in rule for every one).  None changes what is computed; the
   * linear-algebra choices change the rounding only (float64-accurate either way). */
  int32_t autotune;             /* 1 (mixed modes): tks_plan_create times candidate schedules on the
                                   plan's own inputs before returning (lanes, then each knob below,
                                   one at a time from the rule, a second round when the first changed
                                   anything, keeping a candidate only when it is at least 2% faster),
                                   using a scratch workspace and outputs it
                                   allocates and frees; the plan keeps the fastest and reports the
                                   candidates and times through tks_plan_tuning.  Autotuning runs
                                   the recompression several times on a stream of its own and
                                   synchronizes the device. */
  int32_t sketch_qr;            /* TKS_MIXED QR of Y_n: 0 rule (shifted CholeskyQR3 where S_n <= 64
                                   and n_n >= S_n, else Householder), 1 the same, 2 Householder always,
                                   3 CholeskyQR2 where the rule takes CholeskyQR3 (a matrix whose
                                   second pass finds X R^-1 far from orthonormal, any pivot below 1/4
                                   of its diagonal entry, falls back to Householder) */
  int32_t hosvd_r;              /* TKS_MIXED triangular factor of H_(n)^T: 0 rule (shifted CholeskyQR3
                                   for b_n <= 64, else Householder TSQR), 1 the same, 2 TSQR always,
                                   3 CholeskyQR2 as for sketch_qr */
  int32_t proj_chunk;           /* fused order-3 projection: 0 rule (16), else 8 or 16 mode-3
                                   indices per staged chunk at most */
  int32_t tc_stages;            /* tensor-core GEMM shared-memory ring: 0 rule (up to 4 stages as the
                                   operand planes fit), else 2..4 at most */
} tks_params;

typedef struct tks_plan tks_plan;

typedef struct {
  size_t workspace_bytes;       /* device scratch each execute call needs (256-byte aligned) */
  int64_t omega_elems;          /* float64 elements of the Omega buffer (tks_generate_omega) */
  int64_t sketch_elems;         /* float64 elements of the Y buffer (tucker_sum_sketch) */
  int64_t basis_elems;          /* float64 elements of a Q buffer (tks_project_core input) */
  int64_t core_elems;           /* float64 elements of an H buffer (tks_project_core output) */
  int64_t output_elems;         /* float64 elements of the recompression output buffer */
  int32_t num_problems;
  int32_t launches_recompress;  /* kernel launches one tucker_sum_recompress enqueues */
  double flops_lowprec;         /* algorithmic flops of the contraction stages, all problems */
  double flops_fp64;            /* algorithmic flops of QR and ST-HOSVD, all problems */
  int64_t grad_core_elems;      /* float64 elements of the core-gradient buffer (backward) */
  int64_t grad_factor_elems;    /* float64 elements of the factor-gradient buffer (backward) */
  int32_t launches_backward;    /* kernel launches one tks_project_core_backward enqueues (0: none) */
  int32_t pad;
} tks_plan_info_t;

typedef struct {
  int32_t order;
  int32_t R[TKS_MAX_ORDER];              /* sum of term ranks per mode */
  int32_t omega_cols[TKS_MAX_ORDER];     /* s_m: columns of Omega_m */
  int32_t sketch_cols[TKS_MAX_ORDER];    /* S_n: columns of Y_n */
  int32_t basis_cols[TKS_MAX_ORDER];     /* b_n = min(n_n, S_n): columns of Q_n, H's dims */
  int32_t max_ranks[TKS_MAX_ORDER];      /* rmax_n = min(target_n, b_n) */
  int64_t omega_off[TKS_MAX_ORDER];      /* element offsets of Omega_m (n_m x s_m) */
  int64_t sketch_off[TKS_MAX_ORDER];     /* element offsets of Y_n (n_n x S_n) */
  int64_t basis_off[TKS_MAX_ORDER];      /* element offsets of Q_n (n_n x b_n) */
  int64_t core_off;                      /* element offset of H (b_1 x ... x b_d) */
  int64_t out_core_off;                  /* element offset of the output core (rmax_1 x ... ) */
  int64_t out_factor_off[TKS_MAX_ORDER]; /* element offsets of U~_n (n_n x rmax_n) */
  int64_t grad_core_off;                 /* element offset of this problem's packed core gradients */
  int64_t grad_factor_off[TKS_MAX_ORDER];/* element offsets of dUcat_n (n_n x R_n) */
} tks_problem_info_t;

/* Validates the problems, computes sketch sizes (Sec. 3.2: s = max_n ell_n for Khatri-Rao,
 * Eq. heuristic_formula in exact integer form for Kronecker), workspace layout and launch
 * tables, and copies the tables to the current CUDA device.  Host-only apart from those
 * allocations and copies; synchronous.  At most 2^20 problems (TKS_EINVAL above); a plan one of
 * whose launches would count more than 2^31 - 1 tiles or elements is refused with
 * TKS_EUNSUPPORTED (split the batch over several plans).  On error *plan is set to NULL. */
TKS_API tks_status tks_plan_create(tks_plan** plan, const tks_problem* problems, int32_t num_problems,
                           const tks_params* params);

/* The schedule the plan runs, as one JSON object written to buf (host, cap bytes, NUL-terminated,
 * truncated to fit; *len receives the full length without the NUL):
 *   {"autotuned": 0|1, "picked": {knobs}, "rule": {knobs}, "rule_ms": t, "picked_ms": t,
 *    "candidates": [{"knobs": {...}, "ms": t}, ...]}
 * with knobs {"lanes", "sketch_qr", "hosvd_r", "proj_chunk", "tc_stages"} as tks_params takes them
 * (so a caller can create later plans with the picks and autotune = 0).  Times are milliseconds per
 * tucker_sum_recompress measured during tks_plan_create (0 when the plan was not autotuned). */
TKS_API tks_status tks_plan_tuning(const tks_plan* plan, char* buf, int64_t cap, int64_t* len);
TKS_API void tks_plan_destroy(tks_plan* plan);
TKS_API tks_status tks_plan_info(const tks_plan* plan, tks_plan_info_t* info);
TKS_API tks_status tks_problem_info(const tks_plan* plan, int32_t problem, tks_problem_info_t* info);

/* Sketch sizes of one problem without a plan or a device (host-only; the values tks_problem_info
 * reports as omega_cols and sketch_cols for a problem with these targets and oversamplings, so a
 * caller of tucker_sum_sketch_noalloc can size Y_out).  With ell_m = target_ranks[m] +
 * oversampling[m]: Khatri-Rao (Sec. 3.2), s_m = S_m = max_j ell_j; Kronecker, s_m is the least s
 * with (s ell_m)^(d-1) >= prod_j ell_j (the exact integer form of Eq. heuristic_formula, which meets
 * Eq. sketch_condition) and S_m = prod_{j != m} s_j.  order = d; target_ranks, oversampling,
 * omega_cols and sketch_cols are host arrays of d entries (the last two written only on success).
 * TKS_EINVAL for an unknown sketch type, d outside 2..TKS_MAX_ORDER, a NULL pointer, a target below
 * 1, a negative oversampling or an ell_m above 2^21; TKS_EUNSUPPORTED for a Kronecker S_m above
 * 8192 (the limit tks_plan_create applies). */
TKS_API tks_status tks_sketch_sizes(int32_t sketch, int32_t order, const int32_t* target_ranks,
                                    const int32_t* oversampling, int32_t* omega_cols, int32_t* sketch_cols);

/* Writes every Omega_m (n_m x s_m, float64, column-major) of every problem into the device
 * buffer omega_out at the offsets of tks_problem_info.  Draw e = i + n_m c of problem p, mode m
 * is Philox4x64-10 block e/4 under key (seed, 0) and counter (e/4, m, p, 0), turned into normals
 * by Box-Muller (lane e%4).  In TKS_MIXED the values are rounded to float32 then bfloat16.
 * This is the exact Omega every other entry point uses. */
TKS_API tks_status tks_generate_omega(tks_plan* plan, void* workspace, double* omega_out, void* stream);

/* Stages (a) and (b) without the QR: Y_n = sum_k U_k^(n) V_kn (Eqs. KRP_sketch_unfolding /
 * Kron_sketch_unfolding) for every problem and mode, float64, into the device buffer Y_out
 * (layout: tks_problem_info sketch_off; Kronecker column order = first remaining mode fastest). */
TKS_API tks_status tucker_sum_sketch(tks_plan* plan, void* workspace, double* Y_out, void* stream);

/* Stage (c) for given bases: H = sum_k alpha_k G_k x_1 (Q_1^T U_k^(1)) ... x_d (Q_d^T U_k^(d))
 * (Sec. 3.3).  Q_in (device, float64, n_n x b_n per mode at basis_off) is read, H_out (device,
 * float64, b_1 x ... x b_d at core_off) is written. */
TKS_API tks_status tks_project_core(tks_plan* plan, void* workspace, const double* Q_in, double* H_out,
                            void* stream);

/* The whole method: stages (a)-(c) and the ST-HOSVD truncation.  out (device, float64,
 * output_elems) receives per problem the core G~ (rmax_1 x ... x rmax_d at out_core_off) and
 * the factors U~_n = Q_n P_n (n_n x rmax_n at out_factor_off[n]).  ranks_out (device, int32,
 * [num_problems * TKS_MAX_ORDER], entry p*TKS_MAX_ORDER + n) receives the kept ranks r_n <= rmax_n
 * (unused entries 0); entries of the core and
 * columns of U~_n beyond them are zero, so the padded arrays are the same Tucker tensor. */
TKS_API tks_status tucker_sum_recompress(tks_plan* plan, void* workspace, double* out, int32_t* ranks_out,
                                 void* stream);

/* The final truncation alone: ST-HOSVD of given projected cores H (Alg. 2 phase 2; stage 4 of Algs. 3/4),
 * with modes 1..d in order, the rank rule of the plan and U~_n = Q_n P_n.  Q_in (device, float64, the
 * basis layout of tks_project_core) and H_in (device, float64, its core layout) are read; out and
 * ranks_out (device) receive exactly what tucker_sum_recompress writes.  TKS_FP64 and TKS_MIXED plans
 * run it in float64 (TSQR of each unfolding H_(n)^T, one-sided Jacobi SVD of its triangular factor;
 * TKS_MIXED takes the mode products H x_n P_n^T and Q_n P_n float64-accurate on the tensor cores),
 * TKS_MIXED_F32LA in float32. */
TKS_API tks_status tks_truncate_core(tks_plan* plan, void* workspace, const double* Q_in, const double* H_in,
                                     double* out, int32_t* ranks_out, void* stream);

/* Relative truncation error of the ST-HOSVD of the last tucker_sum_recompress (or tks_truncate_core)
 * run with this workspace (Alg. 2, phase 2): per problem, err_out[p] = ||H - H~||_F / ||H||_F with
 * H the projected core and H~ its truncation, from the singular values each mode discarded (the
 * discarded parts of successive modes are orthogonal, so their squared norms add up).  It does not
 * include the sketching error of the bases Q_n.  err_out: device, float64, num_problems entries.
 * Enqueued on `stream` after the recompression; TKS_EINVAL for a null argument. */
TKS_API tks_status tks_truncation_error(tks_plan* plan, void* workspace, double* err_out, void* stream);

/* Backward of the core projection (Sec. 3.3) with the bases held fixed (stop-gradient through Q):
 * with A_kn = Q_n^T U_k^(n) and Hbar = dL/dH given (device, float64, the H layout of
 * tks_project_core), writes
 *   dcores   (device, float64, grad_core_elems): per problem at grad_core_off the cores' packing of
 *            tks_problem.cores, term k holding dL/dG_k = alpha_k Hbar x_1 A_k1^T ... x_d A_kd^T
 *   dfactors (device, float64, grad_factor_elems): per problem and mode at grad_factor_off[n] the
 *            Ucat layout n_n x R_n, term k's columns holding
 *            dL/dU_k^(n) = alpha_k Q_n [ (Hbar x_{j != n} A_kj^T)_(n) G_k,(n)^T ].
 * The A_kn are recomputed from Q_in and the factors (nothing is kept from a forward call).
 * Plans whose problems are all of order 3 (TKS_EUNSUPPORTED otherwise): TKS_FP64 computes in float64
 * on the CUDA cores; the mixed modes run A_n^T = Ucat_n^T Q_n, Hbar x_1 A_0cat^T, Hbar x_3 A_2cat^T and
 * dUcat_n^T = Bcat_n^T Q_n^T as bf16 plane products on the tensor cores (hi/mid/lo splits of the float64
 * and float32 operands, float32 accumulation) and the per-term contractions in float32, writing the
 * same float64 layouts. */
TKS_API tks_status tks_project_core_backward(tks_plan* plan, void* workspace, const double* Q_in,
                                             const double* Hbar_in, double* dcores, double* dfactors,
                                             void* stream);

/* Failure-path controls, for tests and diagnosis.  wait_cycles > 0 bounds every device-side wait of
 * this plan's tensor-core kernels to that many SM clock cycles (0 restores the default, about 2 s at
 * 2 GHz).  stall = 1 makes the copy-issuing thread of each tensor-core GEMM of the plan first wait
 * for a device word that nothing sets, so that its wait runs out: the kernel records TKS_ETIMEOUT,
 * drains its own copies and products (bounded), frees its tensor memory and returns; the launch
 * sequence completes with undefined results and tks_sync_status reports TKS_ETIMEOUT.  stall = 0
 * restores normal operation.  Host-only; applies to calls enqueued afterwards.  TKS_EINVAL for
 * wait_cycles < 0 or stall outside {0, 1}. */
TKS_API tks_status tks_plan_set_fault_test(tks_plan* plan, int64_t wait_cycles, int32_t stall);

/* Synchronizes stream, then returns and clears the first error a kernel of this plan recorded
 * since the previous call (TKS_ENONFINITE, TKS_ENOCONV, TKS_ETIMEOUT), else TKS_OK. */
TKS_API tks_status tks_sync_status(tks_plan* plan, void* stream);

/* Per-stage timing of tucker_sum_recompress with CUDA events recorded on the caller's stream
 * between the plan's launches (no synchronization is added).  tks_profile_begin arms it for
 * the next max_calls calls; tks_profile_end synchronizes on the last recorded event, fills up
 * to cap entries (one per launch of the plan's launch list, in launch order) and disarms it.
 * flops and bytes are the stage's algorithmic counts for one call (all problems): every real
 * multiply-add counts 2 flops; bytes count each operand read once and each result written
 * once (float64 or the operand's own element size). */
typedef struct {
  char name[32];          /* stage, e.g. "b2:Y=UcatVcat" */
  int32_t kind;           /* launch kind: 0 Omega, 1 float64 GEMM, 2 split-K reduction, 3 core sketch,
                             4 QR, 5 float64 TSQR level, 6 tensor-core GEMM, ... (the list in binding.py) */
  int32_t calls;          /* recompress calls timed */
  double ms;              /* summed duration over those calls */
  double flops;           /* algorithmic flops of one call */
  double bytes;           /* algorithmic bytes of one call */
} tks_step_profile_t;

TKS_API tks_status tks_profile_begin(tks_plan* plan, int32_t max_calls);
TKS_API tks_status tks_profile_end(tks_plan* plan, tks_step_profile_t* out, int32_t cap, int32_t* nsteps);

/* The structured sketch of ONE problem (same result as tucker_sum_sketch with TKS_FP64 and that
 * problem alone in a plan) for callers that cannot allocate device memory: code that must not
 * call cudaMalloc because another framework owns all device memory through its own pool, because
 * it runs where allocation is forbidden or too slow (real-time loops, callbacks on a hot path),
 * or because it is embedded in a host program that never creates a plan.  The paper has no
 * counterpart of this entry point; it is a deployment variant of tucker_sum_sketch.
 *
 * Inputs and outputs are the caller's: problem and params as for tks_plan_create (params must be
 * TKS_FP64 with dtype F64; omega_lowprec and lanes are checked as there, and omega_lowprec = 1
 * draws the mixed modes' Omega), Y_out a device buffer of sum_n n_n S_n float64 where Y_n
 * (n_n x S_n, column-major) starts at element sum_{m<n} n_m S_m, S_n being the sketch_cols that
 * tks_problem_info reports for the same problem, or tks_sketch_sizes without a plan (Khatri-Rao:
 * max_m ell_m; Kronecker: the product of the other modes' s_j).  The descriptor tables and the intermediates Omega_j, M_j, Vcat_n live
 * in a static device array of TKS_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
 * until the process exits; a problem needing more is rejected with TKS_EINVAL and a message giving
 * both sizes.  No cudaMalloc, cudaFree or other allocating call is made.  The first call on a
 * device (and the first call after that device's context was destroyed, e.g. by cudaDeviceReset)
 * looks up the array's device address (cudaGetSymbolAddress) for that device; make that first call
 * before any stream capture on that device.  The descriptor
 * tables are copied to the array from host memory that lives only for the duration of the call.
 * Every call reuses the same array and leaves its
 * contents behind; nothing in it needs to start at zero (each element a call reads is written
 * earlier by the same call).  Calls enqueued one after another on one stream are ordered; calls
 * whose work overlaps on a GPU (other streams, other host threads) race on the array: serialize
 * them. */
#define TKS_NOALLOC_SCRATCH_BYTES (8u << 20)
TKS_API tks_status tucker_sum_sketch_noalloc(const tks_problem* problem, const tks_params* params, double* Y_out,
                                             void* stream);

/* ---------------------------------------------------------------------------------------------
 * Effective subrank heuristic (Alg. 5, Sec. 3.2 "Heuristic Subrank Selection"), the step before
 * the sketch sizes of Alg. 3/4 when the ranks come from a tolerance instead of target ranks.
 * For every problem and mode n, in float64:
 *   V_n = [ w_1 U_1^(n), ..., w_K U_K^(n) ],  w_k = |alpha_k| ||G_k||_F
 *   lambda = eigenvalues of V_n^T V_n, clamped at zero, descending
 *   rank_n = min{ r >= 1 : sum_{j > r} lambda_j <= eps^2 / d * sum_j lambda_j }
 *   ell_n = rank_n + p_n
 * The library forms the smaller of V_n^T V_n (R_n x R_n) and V_n V_n^T (n_n x n_n): both have the
 * same nonzero eigenvalues, and the zero ones change no sum of the rule.  The Gram matrix has
 * order m_n = min(n_n, R_n) <= 2048 (TKS_EUNSUPPORTED otherwise).  Sketch sizes follow from ell
 * exactly as in tks_plan_create: a plan whose problems carry target_ranks = ell and
 * oversampling = 0 (with trunc_tol = eps for the final ST-HOSVD) runs Alg. 3/4 as printed.
 *
 * tks_subrank_plan_create reads problems as tks_plan_create does, except that target_ranks is
 * ignored and oversampling gives p_n; of params only dtype (F64 or BF16 cores and factors) and
 * trunc_tol (eps > 0) are used.  Host-only apart from one device allocation for the launch
 * tables and the status word; synchronous.  On error *plan is set to NULL. */
typedef struct tks_subrank_plan tks_subrank_plan;

typedef struct {
  size_t workspace_bytes;       /* device scratch of tks_effective_subrank (256-byte aligned) */
  int64_t eigenvalue_elems;     /* float64 elements of the optional eigenvalue buffer */
  int32_t num_problems;
  int32_t launches;             /* kernel launches one tks_effective_subrank enqueues */
  int32_t max_dim;              /* largest Gram order m over all problems and modes */
  int32_t pad;
  double flops;                 /* algorithmic float64 flops of one call: the Gram matrices
                                   (2 x contraction x m(m+1)/2) and their tridiagonalization
                                   (4/3 m^3) */
} tks_subrank_info_t;

TKS_API tks_status tks_subrank_plan_create(tks_subrank_plan** plan, const tks_problem* problems,
                                           int32_t num_problems, const tks_params* params);
TKS_API void tks_subrank_plan_destroy(tks_subrank_plan* plan);
TKS_API tks_status tks_subrank_info(const tks_subrank_plan* plan, tks_subrank_info_t* info);
/* Per mode of one problem (host arrays of TKS_MAX_ORDER entries, unused modes 0): the Gram order
 * m_n and the element offset of its eigenvalues in the eigenvalue buffer. */
TKS_API tks_status tks_subrank_problem_info(const tks_subrank_plan* plan, int32_t problem, int32_t* dims_out,
                                            int64_t* eig_off_out);
/* Enqueues the heuristic on stream.  ranks_out and ell_out (device, int32, [num_problems *
 * TKS_MAX_ORDER], entry p*TKS_MAX_ORDER + n; entries n >= d are not written) receive rank_n and
 * ell_n.  eigenvalues_out (device, float64, eigenvalue_elems, or NULL) receives each mode's m_n
 * eigenvalues in descending order, unclamped, at the offsets of tks_subrank_problem_info.
 * workspace: workspace_bytes of device memory, 256-byte aligned. */
TKS_API tks_status tks_effective_subrank(tks_subrank_plan* plan, void* workspace, int32_t* ranks_out,
                                         int32_t* ell_out, double* eigenvalues_out, void* stream);
/* Failure-path controls, for tests and diagnosis.  wait_cycles > 0 bounds every device-side wait of
 * this plan's tensor-core kernels to that many SM clock cycles (0 restores the default, about 2 s at
 * 2 GHz).  stall = 1 makes the copy-issuing thread of each tensor-core GEMM of the plan first wait
 * for a device word that nothing sets, so that its wait runs out: the kernel records TKS_ETIMEOUT,
 * drains its own copies and products (bounded), frees its tensor memory and returns; the launch
 * sequence completes with undefined results and tks_sync_status reports TKS_ETIMEOUT.  stall = 0
 * restores normal operation.  Host-only; applies to calls enqueued afterwards.  TKS_EINVAL for
 * wait_cycles < 0 or stall outside {0, 1}. */
TKS_API tks_status tks_plan_set_fault_test(tks_plan* plan, int64_t wait_cycles, int32_t stall);

/* Synchronizes stream, then returns and clears the first error a kernel of this plan recorded
 * (TKS_ENONFINITE for a NaN or Inf in a Gram matrix), else TKS_OK. */
TKS_API tks_status tks_subrank_sync_status(tks_subrank_plan* plan, void* stream);

/* Flops the last tks_effective_subrank call executed (Alg. 5 phase 1, float64): the Gram matrices'
 * 2 c m(m+1)/2 plus, for each matrix, sum_{k < K} 4 (m - k)^2 over the K reduction steps the
 * tridiagonalization ran before its trailing block was numerically zero (K = m - 1 without an early
 * end), so that achieved rates can be stated on the work done rather than the 4/3 m^3 of a full
 * reduction.  Reads a small device array synchronously: call it after tks_subrank_sync_status.
 * *flops (host) receives the count. */
TKS_API tks_status tks_subrank_executed_flops(const tks_subrank_plan* plan, double* flops);

TKS_API const char* tks_last_error(void);
TKS_API const char* tks_status_string(tks_status status);

#ifdef __cplusplus
}
#endif
#endif /* TKS_H */

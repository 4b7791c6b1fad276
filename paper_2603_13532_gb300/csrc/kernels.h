// Launch wrappers of the stage kernels (all asynchronous on `stream`).
#pragma once

#include "tks_internal.h"

namespace tks {

// Gaussian Omega (float64, or bf16-rounded values stored as float64 when job.bf16).
void launch_omega(const OmegaJob* jobs, int njobs, int64_t total_blocks, const Bases& bases,
                  uint64_t seed, cudaStream_t stream);
// Grouped strided float64 GEMM; split-K jobs are finished by launch_splitk_reduce_f64.
void launch_gemm_f64(const GemmJob* jobs, int njobs, int total_tiles, const Bases& bases,
                     cudaStream_t stream);
void launch_splitk_reduce_f64(const GemmJob* jobs, int njobs, int64_t total_elems,
                              const Bases& bases, cudaStream_t stream);
// Khatri-Rao / Kronecker core sketch V_kn (float64).
void launch_core_sketch_f64(const CoreSketchJob* jobs, int njobs, int64_t total, const Bases& bases,
                            cudaStream_t stream);
// Householder QR, one CTA per job.
void launch_qr_f64(const QrJob* jobs, int njobs, const Bases& bases, Status* status,
                   cudaStream_t stream);
// Float64 ST-HOSVD: one TSQR level (each job factors one block of a float64 source into a float64
// triangular factor) and the one-sided Jacobi SVD of the b x b factors, one CTA per job.
int tsqr64_block_rows(int max_cols);     // rows of a block: 256 up to 64 columns, else 128
cudaError_t prepare_la64(int bmax);      // raises the dynamic shared memory limits
void launch_tsqr_f64(const TsqrJob* jobs, int njobs, int max_cols, const Bases& bases, cudaStream_t stream);
void launch_svd_f64(const SvdJob* jobs, int njobs, int bmax, const Bases& bases, Status* status,
                    cudaStream_t stream);
// Float64 mode products with a small matrix (ST-HOSVD truncation and final factors), 64 fibres per CTA.
int ttm64_tiles(int64_t fibres);
// max_cols: the largest rmax among the launch's jobs
void launch_ttm_f64(const TtmJob* jobs, int njobs, int total_tiles, int max_cols, int bmax, const Bases& bases,
                    cudaStream_t stream);

// Tensor-core (tcgen05) grouped GEMM over bf16 planes; maps = device array of CUtensorMap.
// (launch shape: tc_gemm_shape in tc_shape.h)
cudaError_t prepare_tc_gemm();
// wait_cycles bounds every mbarrier wait; stall_word (tests of the timeout path) is a device word that
// nothing sets, waited for by the copy-issuing thread before its first copy, or NULL.  kmax: the
// launch's longest contraction (with total_tiles it sets CTAs per SM and partial accumulators);
// allow_two = false keeps one CTA per SM (launches beside other streams' TMEM-holding kernels).
void launch_tc_gemm(const TcJob* jobs, int njobs, int total_tiles, const void* maps, int na_max, int nb_max,
                    const Bases& bases, Status* status, long long wait_cycles, const int* stall_word,
                    int max_stages, int kmax, bool allow_two, cudaStream_t stream);

// Float32 CUDA-core kernels of the mixed path.
void launch_simt_gemm_f32(const SimtJob* jobs, int njobs, int total_tiles, const Bases& bases,
                          cudaStream_t stream);
void launch_core_sketch_f32(const CoreSketchF32Job* jobs, int njobs, int64_t total, const Bases& bases,
                            cudaStream_t stream);
// Order-3 shared-memory kernels (one CTA per job); smem = bytes of the largest job.
cudaError_t prepare_order3_kernels();
void launch_core_sketch_krp3(const CoreSketchF32Job* jobs, int njobs, size_t smem, const Bases& bases,
                             cudaStream_t stream);
void launch_chain3(const Chain3Job* jobs, int njobs, size_t smem, const Bases& bases, cudaStream_t stream);
// Mode products with a small matrix (128 fibres per CTA).
int ttm_rows_tiles(int64_t rows);
bool ttm_rows_fits(int b, int rmax);
cudaError_t prepare_ttm_rows();
void launch_ttm_rows(const TtmJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream);
// Khatri-Rao core sketches of order-3 terms on the tensor cores, one CTA per term: the dynamic
// shared memory of a term, and whether two such CTAs fit one SM.
size_t sketch3_smem_bytes(const int r[3]);
bool sketch3_two_per_sm(const int r[3]);
cudaError_t prepare_sketch3();
void launch_sketch3(const Sketch3Job* jobs, int njobs, size_t smem, const Bases& bases, Status* status,
                    cudaStream_t stream);
// Khatri-Rao core sketches of order-4 terms, one CTA per term: the core slice kc (mode-1 indices per
// pass) that fits budget_bytes of shared memory, and the dynamic shared memory of a job.
int sketch4_slice(const int r[4], size_t budget_bytes);
size_t sketch4_smem_bytes(const int r[4], int kc);
cudaError_t prepare_sketch4();
void launch_sketch4(const Sketch4Job* jobs, int njobs, size_t smem, const Bases& bases, cudaStream_t stream);
// Fused order-3 projection; `jobs` is followed in memory by the Proj3Term records.
size_t proj3_smem_bytes();
cudaError_t prepare_proj3();
void launch_proj3(const Proj3Job* jobs, int njobs, bool f32_cores, const Bases& bases, Status* status,
                  cudaStream_t stream);
// Order-4 fold G'_k(a1) = alpha_k G_k x_2 A_2k[a1, :], one CTA per (term, i3); smem from fold4_smem_bytes.
size_t fold4_smem_bytes(int r0, int r1, int r2, int b1);
cudaError_t prepare_fold4();
void launch_fold4(const Fold4Job* jobs, int njobs, size_t smem, const Bases& bases, cudaStream_t stream);
void launch_split_f64(const SplitJob* jobs, int njobs, int64_t tiles, const Bases& bases, cudaStream_t stream);
void launch_transpose_bf16(const TransposeJob* jobs, int njobs, int total_tiles, const Bases& bases,
                           cudaStream_t stream);

// Float32 small dense linear algebra (Householder QR, one-sided Jacobi SVD).
void launch_qr_f32(const QrF32Job* jobs, int njobs, const Bases& bases, Status* status, cudaStream_t stream);
cudaError_t prepare_svd_f32(int bmax);
// Householder QR with the matrix resident in shared memory (n * S floats), explicit Q.
size_t qr_smem_bytes(int64_t n, int S);
// Householder QR with Y held in registers (n <= 512, S <= 64), one CTA per job.
bool qr_reg_fits(int64_t n, int S);
size_t qr_reg_smem_bytes(int64_t n, int S);
cudaError_t prepare_qr_reg_f32();
void launch_qr_reg_f32(const QrF32Job* jobs, int njobs, int max_rows, size_t smem, const Bases& bases,
                       Status* status, cudaStream_t stream);
void launch_qr_smem_f32(const QrF32Job* jobs, int njobs, size_t smem, const Bases& bases, Status* status,
                        cudaStream_t stream);
// One TSQR level: each job factors one block of rows and writes its triangular factor.
cudaError_t prepare_tsqr_f32();
// Rows of one TSQR block for factors of at most max_cols columns (512 when the block fits in
// registers with 16 rows per lane, else 256).
int tsqr_block_rows(int max_cols);
void launch_tsqr_f32(const TsqrJob* jobs, int njobs, int max_rows, int max_cols, const Bases& bases,
                     cudaStream_t stream);
void launch_svd_f32(const SvdJob* jobs, int njobs, int bmax, const Bases& bases, Status* status,
                    cudaStream_t stream);

// Float64-accurate mode products on the tensor cores (Ozaki scheme): digit planes of the rows of X
// and of P^T (32 rows per CTA), then one 128 x 64 tile of Y per CTA.
int oz_slice_tiles(int64_t rows);
void launch_oz_slice(const OzSliceJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream);
cudaError_t prepare_oz_gemm();
void launch_oz_gemm(const OzGemmJob* jobs, int njobs, int total_tiles, const void* maps, const Bases& bases,
                    Status* status, long long wait_cycles, cudaStream_t stream);
// Shifted CholeskyQR3 with float64-accurate Gram matrices: column exponents and digit planes of X
// (64-row tiles), G = X^T X (one CTA per job), and the small Cholesky steps (one CTA per job).
int oz_xslice_tiles(int64_t rows);
void launch_oz_xmax(const OzXSliceJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream);
void launch_oz_xdig(const OzXSliceJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream);
void launch_oz_gram(const OzGramJob* jobs, int njobs, const void* maps, const Bases& bases, Status* status,
                    long long wait_cycles, cudaStream_t stream);
void launch_chol_step(const CholJob* jobs, int njobs, const Bases& bases, Status* status, cudaStream_t stream);
// sqrt(sum of the discarded energies / ||H||^2) per problem (one thread each)
void launch_trunc_err(const TruncErrJob* jobs, int njobs, const Bases& bases, cudaStream_t stream);

// Effective subrank heuristic (Alg. 5): term weights, weighted Gram tiles, tridiagonalization
// (one CTA per matrix) and eigenvalues + rank rule (one CTA per matrix).
constexpr int kSubrankMaxDim = 2048;   // largest Gram matrix, m = min(n, R)
void launch_subrank_weights(const WeightJob* jobs, int njobs, const Bases& bases, cudaStream_t stream);
void launch_gram_f64(const GramJob* jobs, int njobs, int total_tiles, const Bases& bases, cudaStream_t stream);
cudaError_t prepare_subrank();
// max_m: the largest m among the jobs of the launch (sizes shared memory and rows per thread)
void launch_tridiag_f64(const SubrankJob* jobs, int njobs, int max_m, const Bases& bases, Status* status,
                        cudaStream_t stream);
void launch_subrank_eig(const SubrankJob* jobs, int njobs, int max_m, const Bases& bases, Status* status,
                        cudaStream_t stream);

}  // namespace tks

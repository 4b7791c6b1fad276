// C ABI of the library: plan creation (validation, sketch sizes, workspace layout, launch
// tables) and the execute entry points, which bind the caller's buffers to the plan's base
// ids and enqueue the prebuilt launches on the caller's stream.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "tks.h"
#include "tks_internal.h"

using namespace tks;

namespace {

thread_local std::string g_last_error;

tks_status fail(tks_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

#define TKS_CUDA_CHECK(call)                                                                  \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(TKS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

constexpr size_t kAlign = 256;
constexpr long long kDefaultWaitCycles = 4000000000LL;   // bound of a device-side wait: about 2 s at 2 GHz
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

Operand op(int32_t base, size_t off_bytes) { return Operand{base, 0, (int64_t)off_bytes}; }
Operand op_abs(const void* p, size_t off_bytes = 0) {
  return Operand{B_ABS, 0, (int64_t)(reinterpret_cast<uintptr_t>(p) + off_bytes)};
}

enum StepKind { S_OMEGA, S_GEMM, S_REDUCE, S_CORESKETCH, S_QR, S_TSQR64, S_TC, S_SIMT, S_CS32, S_SPLIT,
                S_TRANSPOSE, S_QR32, S_SVD32, S_TSQR, S_CS3, S_CHAIN3, S_QRSM, S_PROJ3, S_SK3, S_QRREG, S_TTM,
                S_FOLD4, S_PROJ3F, S_SK3F, S_SK4, S_SVD64, S_TTM64, S_OZSLICE, S_OZGEMM, S_OZXMAX, S_OZGRAM, S_CHOL,
                S_OZXDIG, S_TRUNCERR };

struct Step {
  StepKind kind;
  size_t table_off;   // offset of the job table in the device arena
  int njobs;
  int64_t work;       // tiles / elements / blocks
  char name[32];
  double flops, bytes;
  int na_max = 0, nb_max = 0;   // tensor-core GEMM steps: planes per operand
  int kmax = 0;                 // tensor-core GEMM steps: the longest contraction
  bool beside_lanes = false;    // runs while other lanes' kernels share the GPU (see launch_tc_gemm)
  size_t smem = 0;              // dynamic shared memory of one-CTA-per-job steps
};

Step make_step(StepKind kind, size_t off, int njobs, int64_t work, const char* name, double flops,
               double bytes) {
  Step s;
  s.kind = kind;
  s.table_off = off;
  s.njobs = njobs;
  s.work = work;
  std::snprintf(s.name, sizeof(s.name), "%s", name);
  s.flops = flops;
  s.bytes = bytes;
  return s;
}

// Workspace of shifted CholeskyQR3 of one tall matrix (byte offsets): the two re-formed X, the column
// digit planes and exponents, the Gram matrix, R^-1, the accumulated R, the fallback flag, and the row
// digit planes and exponents of X and of R^-1.
// col, colE: X's column digit planes and column exponents in pass 1; col2, colE2: those of the later
// passes (the same buffers when pass 1's digits need not outlive the factorization)
struct CqBuffers {
  size_t X[2], col, colE, G, Rinv, Racc, flag, rowA, rowAE, rowB, rowBE, part, col2, colE2;
};

struct ProbHost {
  int d = 0, K = 0;
  int64_t n[MAXD] = {};
  int s[MAXD] = {}, S[MAXD] = {}, b[MAXD] = {}, R[MAXD] = {}, rmax[MAXD] = {};
  int target[MAXD] = {}, over[MAXD] = {}, ell[MAXD] = {};
  std::vector<int> ranks;      // K*d
  std::vector<int> roff;       // K*d
  std::vector<int64_t> core_off;
  std::vector<double> alpha;
  const void* cores = nullptr;
  const void* factors[MAXD] = {};
  // element offsets in the caller-visible buffers
  int64_t omega_off[MAXD] = {}, y_off[MAXD] = {}, q_off[MAXD] = {}, h_off = 0;
  int64_t out_core_off = 0, out_fac_off[MAXD] = {};
  // workspace byte offsets
  size_t M[MAXD] = {}, V[MAXD] = {}, W[MAXD] = {}, tau[MAXD] = {}, A[MAXD] = {};
  size_t T = 0, P[MAXD] = {}, ev[MAXD] = {}, theta = 0, Hp[2] = {};
  size_t R64 = 0, stk64[2] = {};   // float64 ST-HOSVD: triangular factor and TSQR stacks
  size_t ozA = 0, ozQ = 0, ozB = 0, ozEA = 0, ozEQ = 0, ozEB = 0;   // TKS_MIXED mode products: digit planes
  size_t cqX[2] = {}, cqCol = 0, cqColE = 0, cqG = 0, cqRinv = 0, cqRacc = 0, cqFlag = 0, cqPart = 0;   // CholeskyQR3
  size_t cqCol2 = 0, cqColE2 = 0, ozB2 = 0, ozEB2 = 0;   // later passes; unscaled P digits for Q_n P_n
  size_t errw = 0;   // ||H||^2 and the discarded energy of every mode (the truncation error estimate)
  CqBuffers qcq[MAXD] = {};   // TKS_MIXED: CholeskyQR3 of the sketches Y_n (flag == 0: Householder QR)
  std::vector<size_t> chain;   // 2 ping-pong buffers per term
  // mixed-precision buffers (bytes): bf16 planes and float32 intermediates
  size_t om_plane[MAXD] = {}, M32[MAXD] = {}, Vp[MAXD][3] = {}, Qp[MAXD][3] = {};
  size_t AT32[MAXD] = {}, ATp[MAXD][3] = {}, Tp[3] = {};
  int ldU[MAXD] = {}, ldV[MAXD] = {}, ldA[MAXD] = {}, ldT = 0;
  bool fused3 = false;   // mixed path: order 3 with b_2, b_3 <= 64 -> fused projection kernel
  bool fused4 = false;   // mixed path: order 4 with b_3, b_4 <= 64 -> fold + fused projection
  size_t g4 = 0;         // workspace of the folded cores G'_k(a1) (float32)
  std::vector<int64_t> g4_off;   // per term: float offset of its b_2 folded cores in g4
  size_t Wh = 0, tauh = 0, R32 = 0, P32[MAXD] = {}, sv[MAXD] = {};   // float32 ST-HOSVD
  size_t stk[2] = {};                                                 // TSQR stacked factors
  // backward of the core projection (order 3, float64)
  size_t bZ0 = 0, bZ2 = 0, bB[MAXD] = {};
  std::vector<size_t> bterm;   // per term: Z01, W1, W0
  // mixed backward: bf16 planes (3 each) of A_n (element (r, a) at a + ldb r), of Hbar with mode 1
  // (resp. mode 3) index fastest, of Bcat_n (element (a, col) at a + ldb col) and of Q_n transposed
  // (element (i, a) at a + ldb i); ldb_n = b_n rounded up to 8
  size_t bAp[MAXD][3] = {}, bHA[3] = {}, bHC[3] = {}, bBp[MAXD][3] = {}, bQT[MAXD][3] = {};
  int ldb[MAXD] = {};
  int64_t gcore_off = 0, gfac_off[MAXD] = {};
  double flops_low = 0.0, flops_f64 = 0.0;
};

struct GemmList {
  std::vector<GemmJob> jobs;
  int64_t tiles = 0;
  int64_t red = 0;
  void add(GemmJob j) {
    if (j.M <= 0 || j.N <= 0 || j.batch <= 0) return;
    if (j.K1 <= 0) j.K1 = std::max(j.K, 1);
    if (j.ksplit < 1) j.ksplit = 1;
    j.kchunk = std::max(16, (ceil_div(std::max(j.K, 1), j.ksplit) + 15) / 16 * 16);
    j.ksplit = std::max(1, ceil_div(std::max(j.K, 1), j.kchunk));
    j.tiles_m = ceil_div(j.M, 64);
    j.tiles_n = ceil_div(j.N, 64);
    j.tile_begin = (int)tiles;   // exact while the launch's total passes the 32-bit check at plan creation
    tiles += (int64_t)j.tiles_m * j.tiles_n * j.batch * j.ksplit;
    j.red_begin = 0;
    if (j.ksplit > 1) {
      j.red_begin = red;
      red += (int64_t)j.batch * j.M * j.N;
    }
    jobs.push_back(j);
  }
};

GemmJob gemm(int M, int N, int K, Operand A, int64_t a_m, int64_t a_k0, Operand B, int64_t b_n,
             int64_t b_k0, Operand C, int64_t c_m, int64_t c_n, double alpha = 1.0) {
  GemmJob j;
  std::memset(&j, 0, sizeof(j));
  j.M = M; j.N = N; j.K = K; j.K1 = K; j.batch = 1; j.ksplit = 1;
  j.A = A; j.a_m = a_m; j.a_k0 = a_k0;
  j.B = B; j.b_n = b_n; j.b_k0 = b_k0;
  j.C = C; j.c_m = c_m; j.c_n = c_n;
  j.alpha = alpha; j.beta = 0.0;
  return j;
}

}  // namespace

struct tks_plan {
  int device = 0;
  tks_params params{};
  int nprob = 0;
  int dmax = 0;
  int bmax = 0;
  std::vector<ProbHost> probs;
  std::vector<char> arena_host;
  char* arena_dev = nullptr;
  Status* status = nullptr;
  size_t ws_bytes = 0;
  size_t ws_omega = 0, ws_Y = 0, ws_Q = 0, ws_H = 0;
  int64_t omega_elems = 0, sketch_elems = 0, basis_elems = 0, core_elems = 0, output_elems = 0;
  std::vector<Step> st_omega, st_sketch, st_project, st_recompress, st_backward, st_truncerr;
  // problems [lane_p0, lane_p1) go into the launch tables being built; with lanes > 1 the
  // recompression has one step list per contiguous group of problems, run on its own stream
  int lane_p0 = 0, lane_p1 = 0;
  std::vector<std::vector<Step>> lane_steps;
  std::vector<cudaStream_t> lane_streams;   // lanes 1..L-1 (lane 0 runs on the caller's stream)
  std::vector<cudaEvent_t> lane_join;       // one per extra lane
  cudaEvent_t lane_fork = nullptr;
  int64_t grad_core_elems = 0, grad_factor_elems = 0;
  bool backward_ok = false;
  // the schedule: knobs as run, and the autotuner's measurements (empty when not autotuned)
  std::string tuning_candidates;
  double tuning_rule_ms = 0.0, tuning_picked_ms = 0.0;
  tks_params tuning_rule{};
  bool autotuned = false;
  std::string build_error;   // set by a table builder that cannot plan a problem
  size_t trunc_from = 0;     // first step of the ST-HOSVD truncation in st_recompress
  // failure-path controls (tks_plan_set_fault_test): the bound of the tensor-core kernels' waits, and
  // whether their copy-issuing thread first waits for a device word that nothing sets
  long long wait_cycles = kDefaultWaitCycles;
  int stall = 0;
  const int* stall_word() const { return reinterpret_cast<const int*>(reinterpret_cast<const char*>(status) + 32); }
  double flops_low = 0.0, flops_f64 = 0.0;

  size_t add_table(const void* p, size_t bytes) {
    const size_t off = align_up(arena_host.size(), 64);
    arena_host.resize(off + bytes);
    std::memcpy(arena_host.data() + off, p, bytes);
    return off;
  }
  // TMA tensor maps of the mixed path: specs at plan time, encoded per workspace pointer
  struct MapSpec {
    int32_t base;
    size_t off;
    uint64_t K, rows, ld;
    uint32_t box_rows;
  };
  std::vector<MapSpec> map_specs;
  std::map<std::tuple<int32_t, size_t, uint64_t, uint64_t, uint64_t, uint32_t>, int> map_index;
  size_t maps_off = 0;
  void* maps_host = nullptr;
  const void* maps_ws = nullptr;
  bool maps_pending = false;
  int map_of(int32_t base, size_t off, uint64_t K, uint64_t rows, uint64_t ld, uint32_t box_rows) {
    auto key = std::make_tuple(base, off, K, rows, ld, box_rows);
    auto it = map_index.find(key);
    if (it != map_index.end()) return it->second;
    const int id = (int)map_specs.size();
    map_specs.push_back(MapSpec{base, off, K, rows, ld, box_rows});
    map_index[key] = id;
    return id;
  }

  // profiling: events recorded around the recompress launches
  int prof_max_calls = 0, prof_calls = 0;
  std::vector<cudaEvent_t> prof_events;

  template <typename T>
  void push(std::vector<Step>& steps, StepKind kind, const std::vector<T>& jobs, int64_t work,
            const char* name, double flops = 0.0, double bytes = 0.0) {
    if (jobs.empty() || work <= 0) return;
    steps.push_back(make_step(kind, add_table(jobs.data(), jobs.size() * sizeof(T)), (int)jobs.size(), work,
                              name, flops, bytes));
  }
  void push_gemm(std::vector<Step>& steps, const GemmList& g, const char* name) {
    if (g.jobs.empty()) return;
    double flops = 0.0, bytes = 0.0;
    for (const auto& j : g.jobs) {
      flops += 2.0 * j.M * j.N * (double)j.K * j.batch;
      bytes += 8.0 * ((double)j.M * j.K + (double)j.K * j.N + (double)j.M * j.N) * j.batch;
    }
    push(steps, S_GEMM, g.jobs, g.tiles, name, flops, bytes);
    std::vector<GemmJob> split;
    for (const auto& j : g.jobs)
      if (j.ksplit > 1) split.push_back(j);
    char rn[32];
    std::snprintf(rn, sizeof(rn), "%s:reduce", name);
    push(steps, S_REDUCE, split, g.red, rn);
  }
  void push_tc(std::vector<Step>& steps, std::vector<TcJob>& jobs, const char* name) {
    if (jobs.empty()) return;
    int64_t tiles = 0;
    int na = 1, nb = 1, kmax = 0;
    double flops = 0.0, bytes = 0.0;
    for (auto& j : jobs) {
      j.tiles_m = ceil_div(j.M, 128);
      j.tiles_n = ceil_div(j.N, 64);
      j.tile_begin = (int)tiles;
      tiles += (int64_t)j.tiles_m * j.tiles_n;
      na = std::max(na, j.na);
      nb = std::max(nb, j.nb);
      kmax = std::max(kmax, (int)j.K);
      flops += 2.0 * j.M * (double)j.N * j.K;
      bytes += 2.0 * ((double)j.M * j.K + (double)j.N * j.K) +
               (double)j.M * j.N * (4.0 * j.epi.has_f32 + 8.0 * j.epi.has_f64 + 2.0 * j.epi.nbf);
    }
    Step st = make_step(S_TC, add_table(jobs.data(), jobs.size() * sizeof(TcJob)), (int)jobs.size(), tiles, name,
                        flops, bytes);
    st.na_max = na;
    st.nb_max = nb;
    st.kmax = kmax;
    steps.push_back(st);
  }
  void push_simt(std::vector<Step>& steps, std::vector<SimtJob>& jobs, const char* name) {
    if (jobs.empty()) return;
    int64_t tiles = 0;
    double flops = 0.0;
    for (auto& j : jobs) {
      j.tiles_m = ceil_div(j.M, 64);
      j.tiles_n = ceil_div(j.N, 64);
      j.tile_begin = (int)tiles;
      tiles += (int64_t)j.tiles_m * j.tiles_n * j.batch;
      flops += 2.0 * j.M * (double)j.N * j.K * j.batch;
    }
    push(steps, S_SIMT, jobs, tiles, name, flops, 0.0);
  }
  void profile_clear() {
    for (auto e : prof_events) cudaEventDestroy(e);
    prof_events.clear();
    prof_max_calls = prof_calls = 0;
  }
};

namespace {

int64_t prod(const int* v, int n) {
  int64_t p = 1;
  for (int i = 0; i < n; ++i) p *= v[i];
  return p;
}

// Largest ell_n = target_n + oversampling_n accepted: it keeps prod_j ell_j of an order-6 problem
// below 2^126 and every Kronecker s_i at most 2^21 + 1, so the sizes below are exact in the
// fixed-width integers of Wide.
constexpr int64_t kMaxEll = int64_t(1) << 21;
// Most terms in one sum and most sums in one plan: every per-mode rank sum, per-plan count and
// byte offset then fits its integer type with room to spare.
constexpr int kMaxTerms = 1 << 20;
constexpr int kMaxProblems = 1 << 20;

// Non-negative integers below 2^256 as eight 32-bit limbs, least significant first (portable: no
// 128-bit or extended floating point types, whose width differs between hosts).  Room for
// prod_j ell_j < 2^126 and for (s ell_i)^(d-1) < (2^22 2^21)^5 = 2^215.
struct Wide {
  uint32_t w[8] = {1, 0, 0, 0, 0, 0, 0, 0};
  void mul(uint32_t m) {
    uint64_t carry = 0;
    for (int k = 0; k < 8; ++k) {
      const uint64_t t = (uint64_t)w[k] * m + carry;
      w[k] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  bool at_least(const Wide& o) const {
    for (int k = 7; k >= 0; --k)
      if (w[k] != o.w[k]) return w[k] > o.w[k];
    return true;
  }
};

// Least s >= 1 with (s ell_i)^(d-1) >= prod_j ell_j: the exact integer form of
// s_i = ceil((prod_j ell_j)^(1/(d-1)) / ell_i) (Eq. heuristic_formula), by bisection on s in
// [1, 2^22]: with every ell_j <= 2^21, s = 2^22 qualifies, since (2^22 ell_i)^(d-1) >=
// ell_i 2^(21 (d-1)) >= prod_j ell_j.
int kron_size(const int* ell, int d, int i) {
  Wide P;
  for (int j = 0; j < d; ++j) P.mul((uint32_t)ell[j]);
  auto enough = [&](uint32_t sz) {
    Wide v;
    for (int t = 0; t < d - 1; ++t) {
      v.mul(sz);
      v.mul((uint32_t)ell[i]);
    }
    return v.at_least(P);
  };
  uint32_t lo = 1, hi = 1u << 22;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (enough(mid)) {
      hi = mid;
    } else {
      lo = mid + 1;
    }
  }
  return (int)lo;
}

// Columns of Omega_m (s) and of Y_m (S) for one problem (Sec. 3.2: s = max_n ell_n for Khatri-Rao;
// Eq. heuristic_formula per mode for Kronecker, S_n = prod_{j != n} s_j).  ell[m] in [1, kMaxEll].
tks_status sketch_sizes(int sketch, int d, const int* ell, int* s, int* S, const std::string& where) {
  for (int m = 0; m < d; ++m) {
    if (sketch == TKS_SKETCH_KRP) {
      int w = 0;
      for (int j = 0; j < d; ++j) w = std::max(w, ell[j]);
      s[m] = w;
    } else {
      s[m] = kron_size(ell, d, m);
    }
  }
  for (int m = 0; m < d; ++m) {
    if (sketch == TKS_SKETCH_KRP) {
      S[m] = s[m];
      continue;
    }
    int64_t w = 1;
    for (int j = 0; j < d; ++j) {
      if (j == m) continue;
      w *= s[j];   // at most 8192 x (2^21 + 1) before the check below ends the loop
      if (w > 8192) return fail(TKS_EUNSUPPORTED, where + "Kronecker sketch wider than 8192 columns");
    }
    S[m] = (int)w;
  }
  return TKS_OK;
}

tks_status validate_and_size(const tks_problem& pr, const tks_params& prm, ProbHost& h, int pidx) {
  const std::string where = "problem " + std::to_string(pidx) + ": ";
  if (pr.order < 2 || pr.order > TKS_MAX_ORDER) return fail(TKS_EINVAL, where + "order out of range");
  if (pr.num_terms < 1) return fail(TKS_EINVAL, where + "num_terms < 1");
  if (pr.num_terms > kMaxTerms) return fail(TKS_EINVAL, where + "num_terms above 2^20");
  if (!pr.dims || !pr.ranks || !pr.target_ranks || !pr.oversampling || !pr.cores || !pr.factors)
    return fail(TKS_EINVAL, where + "null pointer");
  h.d = pr.order;
  h.K = pr.num_terms;
  h.cores = pr.cores;
  for (int m = 0; m < h.d; ++m) {
    h.n[m] = pr.dims[m];
    if (h.n[m] < 1 || h.n[m] > (1 << 24)) return fail(TKS_EINVAL, where + "dimension out of range");
    h.target[m] = pr.target_ranks[m];
    h.over[m] = pr.oversampling[m];
    if (h.target[m] < 1 || h.over[m] < 0) return fail(TKS_EINVAL, where + "bad target/oversampling");
    if ((int64_t)h.target[m] + h.over[m] > kMaxEll)
      return fail(TKS_EINVAL, where + "target + oversampling above 2^21");
    h.ell[m] = h.target[m] + h.over[m];
    if (!pr.factors[m]) return fail(TKS_EINVAL, where + "null factor pointer");
    h.factors[m] = pr.factors[m];
  }
  h.ranks.assign(pr.ranks, pr.ranks + (size_t)h.K * h.d);
  h.roff.assign((size_t)h.K * h.d, 0);
  h.core_off.assign(h.K, 0);
  h.alpha.assign(h.K, 1.0);
  int64_t coff = 0;
  for (int k = 0; k < h.K; ++k) {
    h.core_off[k] = coff;
    int64_t sz = 1;
    for (int m = 0; m < h.d; ++m) {
      const int r = h.ranks[(size_t)k * h.d + m];
      if (r < 1 || r > TKS_MAX_RANK || r > h.n[m]) return fail(TKS_EINVAL, where + "term rank out of range");
      h.roff[(size_t)k * h.d + m] = h.R[m];
      h.R[m] += r;
      sz *= r;
    }
    coff += sz;
    if (pr.alpha) {
      h.alpha[k] = pr.alpha[k];
      if (!std::isfinite(h.alpha[k])) return fail(TKS_EINVAL, where + "non-finite alpha");
    }
  }
  // sketch sizes (Sec. 3.2 / Eq. heuristic_formula)
  const tks_status sst = sketch_sizes(prm.sketch, h.d, h.ell, h.s, h.S, where);
  if (sst != TKS_OK) return sst;
  for (int m = 0; m < h.d; ++m) {
    h.b[m] = (int)std::min<int64_t>(h.n[m], h.S[m]);
    if (h.b[m] > TKS_MAX_BASIS) return fail(TKS_EUNSUPPORTED, where + "basis wider than TKS_MAX_BASIS");
    h.rmax[m] = std::min(h.target[m], h.b[m]);
  }
  (void)prm;
  return TKS_OK;
}

void count_flops(ProbHost& h, int kron) {
  const int d = h.d;
  double low = 0.0, f64 = 0.0;
  for (int m = 0; m < d; ++m) low += 2.0 * h.n[m] * h.R[m] * h.s[m];               // (a)
  for (int k = 0; k < h.K; ++k) {
    const int* r = &h.ranks[(size_t)k * d];
    const double pr = (double)prod(r, d);
    for (int n = 0; n < d; ++n) {                                                  // (b1)
      if (!kron) {
        low += 2.0 * h.s[0] * pr;
      } else {
        double cur = pr;
        for (int j = 0; j < d; ++j) {
          if (j == n) continue;
          low += 2.0 * h.s[j] * cur;
          cur = cur / r[j] * h.s[j];
        }
      }
    }
    double cur = pr;                                                               // (c2)
    for (int t = 0; t + 1 < d; ++t) {
      low += 2.0 * h.b[t] * cur;
      cur = cur / r[t] * h.b[t];
    }
  }
  double Pd = 1;
  for (int j = 0; j + 1 < d; ++j) Pd *= h.b[j];
  for (int n = 0; n < d; ++n) {
    low += 2.0 * h.n[n] * h.R[n] * h.S[n];                                         // (b2)
    low += 2.0 * h.b[n] * h.n[n] * h.R[n];                                         // (c1)
    f64 += 4.0 * h.n[n] * (double)h.b[n] * h.b[n];                                 // QR + Q
  }
  low += 2.0 * h.b[d - 1] * h.R[d - 1] * Pd;                                       // (c3)
  double cur[MAXD];
  for (int j = 0; j < d; ++j) cur[j] = h.b[j];
  for (int n = 0; n < d; ++n) {                                                    // ST-HOSVD
    double rest = 1;
    for (int j = 0; j < d; ++j)
      if (j != n) rest *= cur[j];
    f64 += 2.0 * h.b[n] * h.b[n] * rest + 2.0 * h.b[n] * h.rmax[n] * rest + 2.0 * h.n[n] * h.b[n] * h.rmax[n];
    cur[n] = h.rmax[n];
  }
  h.flops_low = low;
  h.flops_f64 = f64;
}

}  // namespace

namespace {

// Launch lists of shifted CholeskyQR3 for a set of tall matrices X (P x b, b <= 64, element (i = l + L r,
// a) at src[l + L a + L b r]), all run by the same grouped launches: three passes of [column digit
// planes, Gram matrix, Cholesky step, row digit planes of X and R^-1, X <- X R^-1]; the third pass
// ends after its Cholesky step, or with Q = X R^-1 when the caller wants the orthonormal factor.
struct CqLists {
  std::vector<OzXSliceJob> xsl[3];
  std::vector<OzGramJob> gram[3];
  std::vector<CholJob> chol[3];
  std::vector<OzSliceJob> slice[3];
  std::vector<OzGemmJob> gemm[3];
  int64_t xsl_total[3] = {0, 0, 0}, slice_total[3] = {0, 0, 0}, gemm_total[3] = {0, 0, 0};
  double gram_flops = 0.0, gemm_flops[3] = {0.0, 0.0, 0.0}, chol_flops[3] = {0.0, 0.0, 0.0};

  // Rout: where the last pass writes R (B_NONE: not wanted); Qout: where X R^-1 of the last pass goes
  // (B_NONE: no product after the last Cholesky step).  passes = 3: shifted CholeskyQR3; passes = 2:
  // CholeskyQR2 (no shift; for condition numbers below about u^-1/2, a breakdown otherwise).  Returns
  // the fallback flag operand (nonzero: a Cholesky step broke down and the Householder factorization
  // must run for this matrix).
  Operand add(tks_plan* plan, Operand src, int64_t P, int64_t L, int b, const CqBuffers& B, Operand Rout,
              Operand Qout, int passes = 3) {
    const int64_t ldP = (P + 7) / 8 * 8;
    const int ldk = 64;
    const Operand flag = op(B_WS, B.flag);
    const Operand X[3] = {src, op(B_WS, B.X[0]), op(B_WS, B.X[1])};
    for (int pass = 0; pass < passes; ++pass) {
      OzXSliceJob xj;
      std::memset(&xj, 0, sizeof(xj));
      xj.src = X[pass];
      xj.part = op(B_WS, B.part);
      xj.expo = op(B_WS, pass == 0 ? B.colE : B.colE2);
      xj.colP = op(B_WS, pass == 0 ? B.col : B.col2);
      xj.P = P;
      xj.L = L;
      xj.ldP = ldP;
      xj.rows_pad = (P + 7) / 8 * 8;
      xj.b = b;
      xj.tiles = oz_xslice_tiles(P);
      xj.tile_begin = (int)xsl_total[pass];
      xsl_total[pass] += xj.tiles;
      xsl[pass].push_back(xj);
      OzGramJob gj;
      std::memset(&gj, 0, sizeof(gj));
      for (int sl = 0; sl < kOzSlices; ++sl)
        gj.map[sl] = plan->map_of(B_WS, xj.colP.off + (size_t)sl * 64 * ldP * 2, P, b, ldP, 64);
      gj.expo = xj.expo;
      gj.G = op(B_WS, B.G);
      gj.P = P;
      gj.b = b;
      gram[pass].push_back(gj);
      gram_flops += 2.0 * (double)P * b * b;
      CholJob ch;
      std::memset(&ch, 0, sizeof(ch));
      ch.G = gj.G;
      ch.Rinv = op(B_WS, B.Rinv);
      ch.Racc = op(B_WS, B.Racc);
      ch.Rout = Rout;
      ch.fallback = flag;
      ch.xexp = xj.expo;
      ch.P = P;
      ch.b = b;
      ch.pass = pass + 1;
      ch.shift = passes == 3 && pass == 0;
      ch.last = pass == passes - 1;
      // pass 1: any positive pivot.  CholeskyQR3 passes 2, 3: X R1^-1 may have a condition number
      // near u^-1/2, so only near-singular pivots fail.  CholeskyQR2 pass 2: X R1^-1 must already be
      // close to orthonormal (||Q1^T Q1 - I|| <= 0.6 keeps every pivot above 1/4 of its diagonal
      // entry), else one more pass would not restore orthogonality to rounding and the matrix goes to
      // Householder.
      ch.pivot_tol = pass == 0 ? 0.0 : (passes == 3 ? 1e-12 : 0.25);
      chol_flops[pass] += (double)b * b * b;
      chol[pass].push_back(ch);
      if (ch.last && Qout.base == B_NONE) break;
      // the next X (or Q) = X Rinv: X's digits (column exponents, folded into Rinv's rows) and the
      // digits of the columns of Rinv
      auto slice_job = [&](Operand s_src, size_t planes, size_t expo, int64_t rows, int64_t Ls) {
        OzSliceJob sj;
        std::memset(&sj, 0, sizeof(sj));
        sj.kexp = Operand{B_NONE, 0, 0};
        sj.src = s_src;
        sj.planes = op(B_WS, planes);
        sj.expo = op(B_WS, expo);
        sj.rows = rows;
        sj.L = Ls;
        sj.rows_pad = (rows + 7) / 8 * 8;
        sj.K = b;
        sj.ld = ldk;
        sj.tiles = oz_slice_tiles(rows);
        sj.tile_begin = (int)slice_total[pass];
        slice_total[pass] += sj.tiles;
        slice[pass].push_back(sj);
        return sj;
      };
      const OzSliceJob sr = slice_job(ch.Rinv, B.rowB, B.rowBE, b, 1);
      OzGemmJob g;
      std::memset(&g, 0, sizeof(g));
      g.M = (int)P;
      g.N = b;
      g.K = b;
      g.tiles_m = ceil_div(g.M, 128);
      g.tiles_n = 1;
      g.tile_begin = (int)gemm_total[pass];
      gemm_total[pass] += g.tiles_m;
      for (int sl = 0; sl < kOzSlices; ++sl) {
        g.mapA[sl] = gj.map[sl];   // the Gram's column planes, read MN-major
        g.mapB[sl] = plan->map_of(B_WS, sr.planes.off + (size_t)sl * sr.rows_pad * ldk * 2, b, b, ldk, 64);
      }
      g.expA = Operand{B_NONE, 0, 0};
      g.a_mn = 1;
      g.expB = sr.expo;
      g.Y = pass == passes - 1 ? Qout : X[pass + 1];
      g.L = L;
      g.rmax = b;
      gemm[pass].push_back(g);
      gemm_flops[pass] += 2.0 * (double)P * b * b;
    }
    return flag;
  }

  void push(tks_plan* plan, std::vector<Step>& steps, const char* tag) const {
    char nm[32];
    for (int pass = 0; pass < 3; ++pass) {
      if (gram[pass].empty()) break;
      std::snprintf(nm, sizeof(nm), "%s.xmax%d[oz]", tag, pass + 1);
      plan->push(steps, S_OZXMAX, xsl[pass], xsl_total[pass], nm);
      std::snprintf(nm, sizeof(nm), "%s.xdig%d[oz]", tag, pass + 1);
      plan->push(steps, S_OZXDIG, xsl[pass], xsl_total[pass], nm);
      std::snprintf(nm, sizeof(nm), "%s.gram%d[oz]", tag, pass + 1);
      plan->push(steps, S_OZGRAM, gram[pass], (int64_t)gram[pass].size(), nm, gram_flops / 3.0, 0.0);
      std::snprintf(nm, sizeof(nm), "%s.chol%d", tag, pass + 1);
      plan->push(steps, S_CHOL, chol[pass], (int64_t)chol[pass].size(), nm, chol_flops[pass], 0.0);
      if (gemm[pass].empty()) continue;
      std::snprintf(nm, sizeof(nm), "%s.slice%d[oz]", tag, pass + 1);
      plan->push(steps, S_OZSLICE, slice[pass], slice_total[pass], nm);
      std::snprintf(nm, sizeof(nm), "%s.XRinv%d[oz]", tag, pass + 1);
      plan->push(steps, S_OZGEMM, gemm[pass], gemm_total[pass], nm, gemm_flops[pass], 0.0);
    }
  }
};

// Stages (a)-(c) of the mixed-precision path.  bf16 operand planes are laid out K-major for the
// tensor-core GEMMs (TMA tiles of 64 k x 128 rows for A, 64 k x 64 rows for B):
//   a1  Omega_m rounded to bf16 (a plane besides the float64 copy)
//   a2  M_m = Ucat_m^T Omega_m            A = Ucat_m (rows r, k = i)    B = Omega_m (rows c, k = i)
//   a3  V_kn (float32 core sketch) -> Vcat_n as hi/mid/lo planes, element (r, c) at r + ldV c
//   a4  Y_n = Ucat_n Vcat_n               A = Ucat_n^T (rows i, k = r)  B = Vcat_n planes (rows c)
//   a5  Q_n = qr(Y_n) in float64, split into planes
//   a6  A_n^T = Ucat_n^T Q_n              A = Ucat_n (rows r, k = i)    B = Q_n planes (rows a)
//   a7  per-term chains in float32, last step written as planes of Tcat (element (r, J) at r + ldT J)
//   a8  H_(d)^T = Tcat^T A_d^T            A = Tcat planes (rows J)      B = A_d^T planes (rows a)
static void build_mixed_stages(tks_plan* plan, int kron, bool f32la) {
  CqLists qcq;   // TKS_MIXED: Q_n = qr(Y_n) by shifted CholeskyQR3 where n_n >= S_n <= 64
  std::vector<QrF32Job> qr32, qrsm, qrreg;
  bool planes_in_qr = false;   // the register QR of this mode also writes the bf16 planes of Q
  size_t qrsm_smem = 0, qrreg_smem = 0;
  double qrreg_flops = 0.0;
  int64_t qrreg_rows = 0;
  std::vector<CoreSketchF32Job> cs3;
  std::vector<Chain3Job> ch3;
  std::vector<Sketch3Job> sk3, sk3f;   // terms whose CTAs fit one / two per SM
  std::vector<Sketch4Job> sk4;         // order-4 Khatri-Rao terms, one CTA each
  size_t sk4_smem = 0;
  double sk4_flops = 0.0;
  size_t sk3_smem = 0, sk3f_smem = 0;
  double sk3_flops = 0.0, sk3f_flops = 0.0;
  std::vector<Proj3Job> p3, p3f;
  std::vector<Proj3Term> p3terms, p3fterms;
  double p3_flops = 0.0, p3_bytes = 0.0, p3f_flops = 0.0, p3f_bytes = 0.0;
  std::vector<Fold4Job> f4;
  size_t f4_smem = 0;
  double f4_flops = 0.0;
  size_t cs3_smem = 0, ch3_smem = 0;
  double cs3_flops = 0.0, ch3_flops = 0.0;
  constexpr size_t kSmemCap = 200 * 1024;
  constexpr int kChainRows = 8;
  std::vector<OmegaJob> om;
  int64_t om_blocks = 0;
  std::vector<TcJob> tcM, tcY, tcA, tcH;
  std::vector<CoreSketchF32Job> cs;
  int64_t cs_total = 0;
  double cs_flops = 0.0;
  std::vector<QrJob> qr;
  double qr_flops = 0.0, qr_bytes = 0.0;
  std::vector<SplitJob> sp, sp_all;
  int64_t sp_total = 0, sp_all_total = 0;
  std::vector<std::vector<SimtJob>> chain(std::max(1, plan->dmax - 1));
  auto tc_job = [](int M, int N, int K) {
    TcJob j;
    std::memset(&j, 0, sizeof(j));
    j.M = M; j.N = N; j.K = K;
    j.epi.alpha = 1.0f;
    return j;
  };
  for (int p = plan->lane_p0; p < plan->lane_p1; ++p) {
    auto& h = plan->probs[p];
    const int d = h.d;
    for (int m = 0; m < d; ++m) {
      const uint64_t n = h.n[m];
      OmegaJob oj;
      std::memset(&oj, 0, sizeof(oj));
      oj.out = op(B_OMEGA, h.omega_off[m] * 8);
      oj.plane = op(B_WS, h.om_plane[m]);
      oj.has_plane = 1;
      oj.count = h.n[m] * h.s[m];
      oj.begin = om_blocks;
      oj.problem = p;
      oj.mode = m;
      oj.bf16 = 1;
      om_blocks += (oj.count + 3) / 4;
      om.push_back(oj);
      TcJob a2 = tc_job(h.R[m], h.s[m], (int)n);
      a2.na = a2.nb = a2.npairs = 1;
      a2.mapA[0] = plan->map_of(B_ABS, reinterpret_cast<uintptr_t>(h.factors[m]), n, h.R[m], n, 128);
      a2.mapB[0] = plan->map_of(B_WS, h.om_plane[m], n, h.s[m], n, 64);
      a2.epi.has_f32 = 1;
      a2.epi.f32 = op(B_WS, h.M32[m]);
      a2.epi.f32_m = 1;
      a2.epi.f32_n = h.R[m];
      tcM.push_back(a2);
    }
    for (int k = 0; k < h.K; ++k) {
      if (d == 3 && !kron && h.s[0] <= 64) {
        const int* r = &h.ranks[(size_t)k * d];
        if (r[0] <= kSketch3MaxRank && r[1] <= kSketch3MaxRank && r[2] <= kSketch3MaxRank) {
          Sketch3Job j;
          std::memset(&j, 0, sizeof(j));
          j.core = op_abs(h.cores, (size_t)h.core_off[k] * 2);
          for (int m = 0; m < 3; ++m) {
            j.M[m] = op(B_WS, h.M32[m]);
            for (int t = 0; t < 3; ++t) j.V[m][t] = op(B_WS, h.Vp[m][t]);
            j.r[m] = r[m];
            j.roff[m] = h.roff[(size_t)k * d + m];
            j.R[m] = h.R[m];
            j.ldv[m] = h.ldV[m];
          }
          j.s = h.s[0];
          j.alpha = (float)h.alpha[k];
          // three contractions of the core with a Khatri-Rao factor, and the factors' entries
          const double fl = 2.0 * h.s[0] * (3.0 * r[0] * r[1] * r[2]) +
                            (double)h.s[0] * ((double)r[0] * r[1] + (double)r[0] * r[2] + (double)r[1] * r[2]);
          // two launches: the terms whose CTAs fit two per SM, and the rest
          if (sketch3_two_per_sm(r)) {
            sk3f.push_back(j);
            sk3f_smem = std::max(sk3f_smem, sketch3_smem_bytes(r));
            sk3f_flops += fl;
          } else {
            sk3.push_back(j);
            sk3_smem = std::max(sk3_smem, sketch3_smem_bytes(r));
            sk3_flops += fl;
          }
          continue;
        }
      }
      if (d == 4 && !kron && h.s[0] <= 64) {
        const int* r = &h.ranks[(size_t)k * d];
        if (r[0] <= kSketch4MaxRank && r[1] <= kSketch4MaxRank && r[2] <= kSketch4MaxRank &&
            r[3] <= kSketch4MaxRank) {
          Sketch4Job j;
          std::memset(&j, 0, sizeof(j));
          j.core = op_abs(h.cores, (size_t)h.core_off[k] * 2);
          for (int m = 0; m < 4; ++m) {
            j.M[m] = op(B_WS, h.M32[m]);
            for (int t = 0; t < 3; ++t) j.V[m][t] = op(B_WS, h.Vp[m][t]);
            j.r[m] = r[m];
            j.roff[m] = h.roff[(size_t)k * d + m];
            j.R[m] = h.R[m];
            j.ldv[m] = h.ldV[m];
          }
          j.s = h.s[0];
          j.kc = sketch4_slice(r, 40 * 1024);
          j.alpha = (float)h.alpha[k];
          sk4.push_back(j);
          sk4_smem = std::max(sk4_smem, sketch4_smem_bytes(r, j.kc));
          sk4_flops += 2.0 * h.s[0] * 4.0 * r[0] * r[1] * r[2] * r[3];
          continue;
        }
      }
      for (int n = 0; n < d; ++n) {
        CoreSketchF32Job j;
        std::memset(&j, 0, sizeof(j));
        j.core = op_abs(h.cores, (size_t)h.core_off[k] * 2);
        for (int m = 0; m < d; ++m) {
          j.M[m] = op(B_WS, h.M32[m]);
          j.r[m] = h.ranks[(size_t)k * d + m];
          j.roff[m] = h.roff[(size_t)k * d + m];
          j.R[m] = h.R[m];
          j.s[m] = h.s[m];
        }
        for (int t = 0; t < 3; ++t) j.V[t] = op(B_WS, h.Vp[n][t]);
        j.d = d;
        j.n = n;
        j.kron = kron;
        j.ldv = h.ldV[n];
        j.S = h.S[n];
        j.alpha = (float)h.alpha[k];
        j.count = (int64_t)j.r[n] * j.S;
        double other = 1.0;
        for (int m = 0; m < d; ++m)
          if (m != n) other *= j.r[m];
        // core_sketch_krp3 layout: M1, M2, V (rows padded to 8) in float32, core in bf16 (rows padded)
        const int rnp = (j.r[n] + 7) / 8 * 8;
        const size_t smem3 = d == 3 ? (size_t)j.S * 4 * (j.r[0] + j.r[1] + j.r[2] - j.r[n] + rnp) +
                                          (size_t)2 * rnp * (j.r[0] * j.r[1] * j.r[2] / j.r[n]) + 16
                                    : 0;
        if (d == 3 && !kron && smem3 <= kSmemCap) {
          cs3.push_back(j);
          cs3_smem = std::max(cs3_smem, smem3);
          cs3_flops += 2.0 * (double)j.count * other;
          continue;
        }
        cs_flops += 2.0 * (double)j.count * other;
        j.begin = cs_total;
        cs_total += j.count;
        cs.push_back(j);
      }
    }
    for (int n = 0; n < d; ++n) {
      const uint64_t nn = h.n[n];
      TcJob a4 = tc_job((int)nn, h.S[n], h.R[n]);
      a4.na = 1;
      a4.nb = 3;
      a4.npairs = 3;
      // A = Ucat_n as the caller stores it (row index fastest), read MN-major: no transposed copy
      a4.mapA[0] = plan->map_of(B_ABS, reinterpret_cast<uintptr_t>(h.factors[n]), nn, h.R[n], nn, 64);
      a4.a_mn = 1;
      for (int t = 0; t < 3; ++t) {
        a4.mapB[t] = plan->map_of(B_WS, h.Vp[n][t], h.R[n], h.S[n], h.ldV[n], 64);
        a4.pa[t] = 0;
        a4.pb[t] = (uint8_t)t;
      }
      a4.epi.has_f64 = 1;
      a4.epi.f64 = op(B_Y, h.y_off[n] * 8);
      a4.epi.f64_m = 1;
      a4.epi.f64_n = (int64_t)nn;
      tcY.push_back(a4);
      if (f32la) {
        QrF32Job q;
        std::memset(&q, 0, sizeof(q));
        q.src = op(B_Y, h.y_off[n] * 8);
        q.src_type = T_F64;
        q.W = op(B_WS, h.W[n]);
        q.tau = op(B_WS, h.tau[n]);
        q.Q = op(B_Q, h.q_off[n] * 8);
        q.want_q = 1;
        q.b = h.b[n];
        q.rows = (int64_t)nn;
        q.cols = h.S[n];
        q.L0 = (int64_t)nn;
        q.s0 = 1;
        q.s1 = 0;
        q.sc = (int64_t)nn;
        const size_t sm = qr_smem_bytes((int64_t)nn, h.S[n]);
        if (qr_reg_fits((int64_t)nn, h.S[n])) {
          qrreg_flops += 4.0 * (double)nn * h.b[n] * h.b[n];
          q.nplanes = 3;
          for (int t = 0; t < 3; ++t) q.Qp[t] = op(B_WS, h.Qp[n][t]);
          planes_in_qr = true;
          qrreg.push_back(q);
          qrreg_smem = std::max(qrreg_smem, qr_reg_smem_bytes((int64_t)nn, h.S[n]));
          qrreg_rows = std::max<int64_t>(qrreg_rows, (int64_t)nn);
        } else if (sm <= 216 * 1024) {
          qrsm.push_back(q);
          qrsm_smem = std::max(qrsm_smem, sm);
        } else {
          qr32.push_back(q);
        }
      } else {
        QrJob q;
        std::memset(&q, 0, sizeof(q));
        q.Y = op(B_Y, h.y_off[n] * 8);
        q.W = op(B_WS, h.W[n]);
        q.Q = op(B_Q, h.q_off[n] * 8);
        q.tau = op(B_WS, h.tau[n]);
        q.gate = Operand{B_NONE, 0, 0};
        q.n = (int)nn;
        q.S = h.S[n];
        q.b = h.b[n];
        if (h.qcq[n].flag) {
          // Q_n by shifted CholeskyQR3 (float64-accurate Grams and products on the tensor cores);
          // the Householder QR runs only if a Cholesky step breaks down (a rank-deficient sketch)
          q.gate = qcq.add(plan, op(B_Y, h.y_off[n] * 8), (int64_t)nn, (int64_t)nn, h.S[n], h.qcq[n], Operand{B_NONE, 0, 0},
                           op(B_Q, h.q_off[n] * 8), plan->params.sketch_qr == 3 ? 2 : 3);
        }
        qr.push_back(q);
      }
      qr_flops += 4.0 * (double)nn * h.b[n] * h.b[n];
      qr_bytes += 8.0 * (double)nn * (h.S[n] + h.b[n]);
      // Q -> bf16 planes: always when Q is given (tks_project_core); in the recompression only
      // where the QR kernel did not write them itself
      SplitJob sj;
      std::memset(&sj, 0, sizeof(sj));
      sj.src = op(B_Q, h.q_off[n] * 8);
      for (int t = 0; t < 3; ++t) sj.dst[t] = op(B_WS, h.Qp[n][t]);
      sj.rows = (int64_t)nn;
      sj.cols = h.b[n];
      sj.ld_src = sj.ld_dst = (int64_t)nn;
      sj.count = sj.rows * sj.cols;
      sj.begin = 0;
      sj.tile_begin = (int32_t)sp_all_total;
      sp_all_total += (sj.count + kSplitTile - 1) / kSplitTile;
      sp_all.push_back(sj);
      if (!planes_in_qr) {
        sj.tile_begin = (int32_t)sp_total;
        sp_total += (sj.count + kSplitTile - 1) / kSplitTile;
        sp.push_back(sj);
      }
      planes_in_qr = false;
      TcJob a6 = tc_job(h.R[n], h.b[n], (int)nn);
      a6.na = 1;
      a6.nb = 3;
      a6.npairs = 3;
      a6.mapA[0] = plan->map_of(B_ABS, reinterpret_cast<uintptr_t>(h.factors[n]), nn, h.R[n], nn, 128);
      for (int t = 0; t < 3; ++t) {
        a6.mapB[t] = plan->map_of(B_WS, h.Qp[n][t], nn, h.b[n], nn, 64);
        a6.pa[t] = 0;
        a6.pb[t] = (uint8_t)t;
      }
      a6.epi.has_f32 = 1;
      a6.epi.f32 = op(B_WS, h.AT32[n]);
      a6.epi.f32_m = 1;
      a6.epi.f32_n = h.R[n];
      if (n == d - 1 && !h.fused3 && !h.fused4) {
        a6.epi.nbf = 3;
        for (int t = 0; t < 3; ++t) a6.epi.bf[t] = op(B_WS, h.ATp[n][t]);
        a6.epi.bf_m = 1;
        a6.epi.bf_n = h.ldA[n];
      }
      tcA.push_back(a6);
    }
    if (h.fused3) {
      // (c2 + c3) fused: one CTA per kProj3Rows mode-1 rows of H
      const int tb = (int)p3terms.size();
      for (int k = 0; k < h.K; ++k) {
        const int* r = &h.ranks[(size_t)k * d];
        Proj3Term t;
        std::memset(&t, 0, sizeof(t));
        t.core = op_abs(h.cores, (size_t)h.core_off[k] * 2);
        for (int q = 0; q < 3; ++q) {
          t.r[q] = r[q];
          t.roff[q] = h.roff[(size_t)k * d + q];
        }
        t.alpha = (float)h.alpha[k];
        t.chunk = proj3_chunk(t.r, 2);
        if (plan->params.proj_chunk > 0) t.chunk = std::min(t.chunk, plan->params.proj_chunk);
        p3terms.push_back(t);
        p3_flops += 2.0 * h.b[0] * ((double)r[0] * r[1] * r[2] + (double)h.b[1] * r[1] * r[2] +
                                    (double)h.b[1] * h.b[2] * r[2]);
      }
      for (int x0 = 0; x0 < h.b[0]; x0 += kProj3Rows) {
        Proj3Job j;
        std::memset(&j, 0, sizeof(j));
        for (int q = 0; q < 3; ++q) {
          j.AT[q] = op(B_WS, h.AT32[q]);
          j.R[q] = h.R[q];
          j.b[q] = h.b[q];
        }
        j.H = op(B_H, h.h_off * 8);
        j.x0 = x0;
        j.rows = std::min(kProj3Rows, h.b[0] - x0);
        j.term_begin = tb;
        j.nterms = h.K;
        j.hs1 = h.b[0];
        j.hs2 = (int64_t)h.b[0] * h.b[1];
        p3.push_back(j);
      }
      p3_bytes += 8.0 * (double)h.b[0] * h.b[1] * h.b[2];
      continue;
    }
    if (h.fused4) {
      // fold mode 2 into the cores: G'_k(a1) = alpha_k G_k x_2 A_2k[a1, :] for every a1 < b_2,
      // then H[:, a1, :, :] is the order-3 projection of the G'_k(a1) (modes 1, 3, 4)
      const int b0 = h.b[0], b1 = h.b[1], b2 = h.b[2], b3 = h.b[3];
      for (int k = 0; k < h.K; ++k) {
        const int* r = &h.ranks[(size_t)k * d];
        for (int i3 = 0; i3 < r[3]; ++i3) {
          Fold4Job f;
          std::memset(&f, 0, sizeof(f));
          f.core = op_abs(h.cores, (size_t)h.core_off[k] * 2);
          f.AT1 = op(B_WS, h.AT32[1]);
          f.out = op(B_WS, h.g4 + (size_t)h.g4_off[k] * 4);
          for (int q = 0; q < 4; ++q) f.r[q] = r[q];
          f.R1 = h.R[1];
          f.roff1 = h.roff[(size_t)k * d + 1];
          f.b1 = b1;
          f.alpha = (float)h.alpha[k];
          f.i3 = i3;
          f4.push_back(f);
          f4_smem = std::max(f4_smem, fold4_smem_bytes(r[0], r[1], r[2], b1));
        }
        f4_flops += 2.0 * b1 * (double)r[0] * r[1] * r[2] * r[3];
      }
      for (int a1 = 0; a1 < b1; ++a1) {
        const int tb = (int)p3fterms.size();
        for (int k = 0; k < h.K; ++k) {
          const int* r = &h.ranks[(size_t)k * d];
          Proj3Term t;
          std::memset(&t, 0, sizeof(t));
          const int64_t blk = (int64_t)r[0] * r[2] * r[3];
          t.core = op(B_WS, h.g4 + (size_t)(h.g4_off[k] + blk * a1) * 4);
          const int modes[3] = {0, 2, 3};
          for (int q = 0; q < 3; ++q) {
            t.r[q] = r[modes[q]];
            t.roff[q] = h.roff[(size_t)k * d + modes[q]];
          }
          t.alpha = 1.0f;
          t.chunk = proj3_chunk(t.r, 4);
          if (plan->params.proj_chunk > 0) t.chunk = std::min(t.chunk, plan->params.proj_chunk);
          p3fterms.push_back(t);
          p3f_flops += 2.0 * b0 * ((double)r[0] * r[2] * r[3] + (double)b2 * r[2] * r[3] + (double)b2 * b3 * r[3]);
        }
        for (int x0 = 0; x0 < b0; x0 += kProj3Rows) {
          Proj3Job j;
          std::memset(&j, 0, sizeof(j));
          const int modes[3] = {0, 2, 3};
          for (int q = 0; q < 3; ++q) {
            j.AT[q] = op(B_WS, h.AT32[modes[q]]);
            j.R[q] = h.R[modes[q]];
            j.b[q] = h.b[modes[q]];
          }
          j.H = op(B_H, (h.h_off + (int64_t)b0 * a1) * 8);
          j.x0 = x0;
          j.rows = std::min(kProj3Rows, b0 - x0);
          j.term_begin = tb;
          j.nterms = h.K;
          j.hs1 = (int64_t)b0 * b1;
          j.hs2 = (int64_t)b0 * b1 * b2;
          p3f.push_back(j);
        }
      }
      p3f_bytes += 8.0 * (double)b0 * b1 * b2 * b3;
      continue;
    }
    // (c2) chains in float32; A_t^T block of term k: element (j, i) at (roff + i) + R_t j
    for (int k = 0; k < h.K; ++k) {
      const int* r = &h.ranks[(size_t)k * d];
      const int rd_off = h.roff[(size_t)k * d + d - 1];
      if (d == 3) {
        const size_t smem = 4 * ((size_t)kChainRows * r[0] + (size_t)r[1] * h.b[1] + (size_t)r[2] * kChainRows * r[1]) +
                            (size_t)2 * r[0] * r[1] * r[2];
        if (smem <= kSmemCap) {
          for (int a0 = 0; a0 < h.b[0]; a0 += kChainRows) {
            Chain3Job c;
            std::memset(&c, 0, sizeof(c));
            c.core = op_abs(h.cores, (size_t)h.core_off[k] * 2);
            c.AT[0] = op(B_WS, h.AT32[0]);
            c.AT[1] = op(B_WS, h.AT32[1]);
            for (int q = 0; q < 3; ++q) {
              c.T[q] = op(B_WS, h.Tp[q]);
              c.r[q] = r[q];
              c.roff[q] = h.roff[(size_t)k * d + q];
            }
            c.R[0] = h.R[0];
            c.R[1] = h.R[1];
            c.b[0] = h.b[0];
            c.b[1] = h.b[1];
            c.a0 = a0;
            c.rows = std::min(kChainRows, h.b[0] - a0);
            c.ldT = h.ldT;
            c.alpha = (float)h.alpha[k];
            ch3.push_back(c);
          }
          ch3_smem = std::max(ch3_smem, smem);
          ch3_flops += 2.0 * h.b[0] * (double)r[0] * r[1] * r[2] + 2.0 * h.b[0] * (double)h.b[1] * r[1] * r[2];
          continue;
        }
      }
      for (int t = 0; t + 1 < d; ++t) {
        int64_t L = 1, Rr = 1;
        for (int j = 0; j < t; ++j) L *= h.b[j];
        for (int j = t + 1; j < d; ++j) Rr *= r[j];
        const int I = r[t], Jn = h.b[t], Rt = h.R[t];
        SimtJob j;
        std::memset(&j, 0, sizeof(j));
        const Operand X = (t == 0) ? op_abs(h.cores, (size_t)h.core_off[k] * 2)
                                   : op(B_WS, h.chain[2 * k + ((t - 1) & 1)]);
        const int32_t xt = (t == 0) ? T_BF16 : T_F32;
        const Operand Ablk = op(B_WS, h.AT32[t] + (size_t)h.roff[(size_t)k * d + t] * 4);
        const bool last = (t == d - 2);
        j.batch = 1;
        j.alpha = (t == 0) ? (float)h.alpha[k] : 1.0f;
        if (L == 1) {
          j.M = Jn; j.N = (int)Rr; j.K = I; j.K1 = I;
          j.A = Ablk; j.a_type = T_F32; j.a_m = Rt; j.a_k0 = 1;
          j.B = X; j.b_type = xt; j.b_n = I; j.b_k0 = 1;
          j.c_m = last ? h.ldT : 1;
          j.c_n = last ? 1 : Jn;
        } else {
          j.M = (int)L; j.N = Jn; j.K = I; j.K1 = I; j.batch = (int)Rr;
          j.A = X; j.a_type = xt; j.a_m = 1; j.a_k0 = L; j.a_b = L * I;
          j.B = Ablk; j.b_type = T_F32; j.b_n = Rt; j.b_k0 = 1;
          j.c_m = last ? h.ldT : 1;
          j.c_n = last ? (int64_t)h.ldT * L : L;
          j.c_b = last ? 1 : L * Jn;
        }
        if (last) {
          j.nbf = 3;
          for (int q = 0; q < 3; ++q) j.cb[q] = op(B_WS, h.Tp[q] + (size_t)rd_off * 2);
        } else {
          j.has_c32 = 1;
          j.c32 = op(B_WS, h.chain[2 * k + (t & 1)]);
        }
        chain[t].push_back(j);
      }
    }
    // (c3) H_(d)^T = Tcat^T A_d^T, six plane products (hi/mid/lo x hi/mid/lo up to second order)
    int64_t Pd = 1;
    for (int j = 0; j + 1 < d; ++j) Pd *= h.b[j];
    const int Rd = h.R[d - 1], bd = h.b[d - 1];
    TcJob c3 = tc_job((int)Pd, bd, Rd);
    c3.na = c3.nb = 3;
    for (int t = 0; t < 3; ++t) {
      c3.mapA[t] = plan->map_of(B_WS, h.Tp[t], Rd, Pd, h.ldT, 128);
      c3.mapB[t] = plan->map_of(B_WS, h.ATp[d - 1][t], Rd, bd, h.ldA[d - 1], 64);
    }
    const uint8_t pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
    c3.npairs = 6;
    for (int t = 0; t < 6; ++t) {
      c3.pa[t] = pa[t];
      c3.pb[t] = pb[t];
    }
    c3.epi.has_f64 = 1;
    c3.epi.f64 = op(B_H, h.h_off * 8);
    c3.epi.f64_m = 1;
    c3.epi.f64_n = Pd;
    tcH.push_back(c3);
  }
  plan->push(plan->st_omega, S_OMEGA, om, om_blocks, "a1:omega", 0.0, 10.0 * plan->omega_elems);
  plan->push(plan->st_sketch, S_OMEGA, om, om_blocks, "a1:omega", 0.0, 10.0 * plan->omega_elems);

  plan->push_tc(plan->st_sketch, tcM, "a2:M=UcatT.Omega[tc]");
  plan->push(plan->st_sketch, S_CS32, cs, cs_total, "a3:core_sketch[f32]", cs_flops, 0.0);
  if (!cs3.empty()) {
    plan->push(plan->st_sketch, S_CS3, cs3, (int64_t)cs3.size(), "a3:core_sketch3[f32]", cs3_flops, 0.0);
    plan->st_sketch.back().smem = cs3_smem;
  }
  if (!sk4.empty()) {
    plan->push(plan->st_sketch, S_SK4, sk4, (int64_t)sk4.size(), "a3:sketch4[f32]", sk4_flops, 0.0);
    plan->st_sketch.back().smem = sk4_smem;
  }
  if (!sk3f.empty()) {
    plan->push(plan->st_sketch, S_SK3F, sk3f, (int64_t)sk3f.size(), "a3:sketch3[tc]", sk3f_flops, 0.0);
    plan->st_sketch.back().smem = sk3f_smem;
  }
  if (!sk3.empty()) {
    plan->push(plan->st_sketch, S_SK3, sk3, (int64_t)sk3.size(), "a3:sketch3b[tc]", sk3_flops, 0.0);
    plan->st_sketch.back().smem = sk3_smem;
  }
  plan->push_tc(plan->st_sketch, tcY, "a4:Y=Ucat.Vcat[tc]");
  plan->push(plan->st_project, S_SPLIT, sp_all, sp_all_total, "a6:Q->planes", 0.0, 14.0 * kSplitTile * sp_all_total);
  const size_t project_from = plan->st_project.size();   // the recompression takes its own split
  plan->push_tc(plan->st_project, tcA, "a6:AT=UcatT.Q[tc]");
  for (size_t t = 0; t < chain.size(); ++t) {
    char nm[32];
    std::snprintf(nm, sizeof(nm), "a7:chain%d[f32]", (int)t);
    plan->push_simt(plan->st_project, chain[t], nm);
  }
  if (!ch3.empty()) {
    plan->push(plan->st_project, S_CHAIN3, ch3, (int64_t)ch3.size(), "a7:chain3[f32]", ch3_flops, 0.0);
    plan->st_project.back().smem = ch3_smem;
  }
  plan->push_tc(plan->st_project, tcH, "a8:H=Tcat.AT[tc]");
  // fused projections: one table each, the jobs followed by the term records they index
  auto push_proj = [&](StepKind kind, const std::vector<Proj3Job>& jobs, const std::vector<Proj3Term>& terms,
                       const char* name, double flops, double bytes) {
    if (jobs.empty()) return;
    std::vector<char> blob(jobs.size() * sizeof(Proj3Job) + terms.size() * sizeof(Proj3Term));
    std::memcpy(blob.data(), jobs.data(), jobs.size() * sizeof(Proj3Job));
    if (!terms.empty())
      std::memcpy(blob.data() + jobs.size() * sizeof(Proj3Job), terms.data(), terms.size() * sizeof(Proj3Term));
    plan->st_project.push_back(make_step(kind, plan->add_table(blob.data(), blob.size()), (int)jobs.size(),
                                         (int64_t)jobs.size(), name, flops, bytes));
    plan->st_project.back().smem = proj3_smem_bytes();
  };
  push_proj(S_PROJ3, p3, p3terms, "a7:project3[f32]", p3_flops, p3_bytes);
  if (!f4.empty()) {
    plan->push(plan->st_project, S_FOLD4, f4, (int64_t)f4.size(), "a7:fold4[f32]", f4_flops, 0.0);
    plan->st_project.back().smem = f4_smem;
  }
  push_proj(S_PROJ3F, p3f, p3fterms, "a7:project4[f32]", p3f_flops, p3f_bytes);
  plan->st_recompress = plan->st_sketch;
  qcq.push(plan, plan->st_recompress, "a5:cq");
  plan->push(plan->st_recompress, S_QR, qr, (int64_t)qr.size(), "a5:qr", qcq.gram[0].empty() ? qr_flops : 0.0,
             qr_bytes);
  plan->push(plan->st_recompress, S_QR32, qr32, (int64_t)qr32.size(), "a5:qr[f32]", qr_flops, qr_bytes);
  if (!qrreg.empty()) {
    // work = the largest row count (selects the kernel's rows per lane)
    plan->push(plan->st_recompress, S_QRREG, qrreg, qrreg_rows, "a5:qr_reg[f32]", qrreg_flops, 0.0);
    plan->st_recompress.back().smem = qrreg_smem;
  }
  if (!qrsm.empty()) {
    plan->push(plan->st_recompress, S_QRSM, qrsm, (int64_t)qrsm.size(), "a5:qr_smem[f32]", qr_flops - qrreg_flops,
               0.0);
    plan->st_recompress.back().smem = qrsm_smem;
  }
  plan->push(plan->st_recompress, S_SPLIT, sp, sp_total, "a6:Q->planes", 0.0, 14.0 * kSplitTile * sp_total);
  for (size_t i = project_from; i < plan->st_project.size(); ++i) plan->st_recompress.push_back(plan->st_project[i]);
}

// ST-HOSVD of H in float32 (Alg. 2 phase 2, modes 1..d in order): per mode, Householder QR of
// H_(n)^T (rows = the other modes, two-level index), one-sided Jacobi SVD of its b x b triangular
// factor (right singular vectors = left singular vectors of H_(n)), rank rule, then
// H <- H x_n P_n^T and U~_n = Q_n P_n on CUDA cores.
static void build_hosvd_f32(tks_plan* plan) {
  for (int n = 0; n < plan->dmax; ++n) {
    std::vector<std::vector<TsqrJob>> tsqr;
    std::vector<SvdJob> svds;
    std::vector<SimtJob> ttm, fac;
    std::vector<TtmJob> ttm2, fac2;
    int64_t ttm_tiles = 0, fac_tiles = 0;
    double ttm_flops = 0.0, fac_flops = 0.0;
    double qflops = 0.0;
    for (int p = plan->lane_p0; p < plan->lane_p1; ++p) {
      auto& h = plan->probs[p];
      const int d = h.d;
      if (n >= d) continue;
      int64_t L = 1, Rr = 1;
      for (int j = 0; j < n; ++j) L *= h.rmax[j];
      for (int j = n + 1; j < d; ++j) Rr *= h.b[j];
      const int b = h.b[n], rmax = h.rmax[n];
      const Operand X = (n == 0) ? op(B_H, h.h_off * 8) : op(B_WS, h.Hp[(n - 1) & 1]);
      const int32_t xt = (n == 0) ? T_F64 : T_F32;
      // TSQR of H_(n)^T (rows = L Rr with the two-level index (l, rr), cols = b): level 0 reads
      // H, later levels read the stacked b x b factors, the last level writes R32
      {
        int64_t rows = L * Rr;
        qflops += 2.0 * (double)rows * b * b;
        Operand src = X;
        int32_t stype = xt;
        int64_t L0 = L, s0 = 1, s1 = L * b, sc = L;
        for (int lvl = 0;; ++lvl) {
          const int nblk = std::max(1, ceil_div(rows, tsqr_block_rows(plan->bmax)));
          const int brows = ceil_div(rows, nblk);
          if (nblk > 1 && (int64_t)nblk * b >= rows) {   // blocks of at least 2b rows always shrink
            plan->build_error = "TSQR levels do not shrink";
            return;
          }
          const bool final_level = (nblk == 1);
          const Operand dst = final_level ? op(B_WS, h.R32) : op(B_WS, h.stk[lvl & 1]);
          const int64_t dst_ld = final_level ? b : (int64_t)nblk * b;
          if ((int)tsqr.size() <= lvl) tsqr.resize(lvl + 1);
          for (int i = 0; i < nblk; ++i) {
            TsqrJob t;
            std::memset(&t, 0, sizeof(t));
            t.src = src;
            t.src_type = stype;
            t.row_begin = (int64_t)i * brows;
            t.rows = (int)std::min<int64_t>(brows, rows - t.row_begin);
            t.cols = b;
            t.L0 = L0;
            t.s0 = s0;
            t.s1 = s1;
            t.sc = sc;
            t.dst = dst;
            t.dst_row0 = (int64_t)i * b;
            t.dst_ld = dst_ld;
            tsqr[lvl].push_back(t);
          }
          if (final_level) break;
          src = dst;
          stype = T_F32;
          rows = (int64_t)nblk * b;
          L0 = rows;
          s0 = 1;
          s1 = 0;
          sc = dst_ld;
        }
      }
      SvdJob sj;
      std::memset(&sj, 0, sizeof(sj));
      sj.R = op(B_WS, h.R32);
      sj.P = op(B_WS, h.P32[n]);
      sj.sv = op(B_WS, h.sv[n]);
      sj.theta = op(B_WS, h.theta);
      sj.rank = op(B_RANKS, (size_t)(p * TKS_MAX_ORDER + n) * 4);
      sj.b = b;
      sj.rmax = rmax;
      sj.first_mode = (n == 0);
      sj.mode = n;
      sj.err = op(B_WS, h.errw);
      sj.order = d;
      sj.tol = plan->params.trunc_tol;
      svds.push_back(sj);
      if (ttm_rows_fits(b, rmax)) {
        // H x_n P^T and Q_n P with the fibre kernel
        TtmJob tj;
        std::memset(&tj, 0, sizeof(tj));
        tj.X = X;
        tj.x_type = xt;
        tj.P = op(B_WS, h.P32[n]);
        tj.L = L;
        tj.Rr = Rr;
        tj.b = b;
        tj.rmax = rmax;
        if (n == d - 1) {
          tj.Y = op(B_OUT, h.out_core_off * 8);
          tj.y_type = T_F64;
        } else {
          tj.Y = op(B_WS, h.Hp[n & 1]);
          tj.y_type = T_F32;
        }
        tj.tiles = ttm_rows_tiles(L * Rr);
        tj.tile_begin = (int)ttm_tiles;
        ttm_tiles += tj.tiles;
        ttm2.push_back(tj);
        ttm_flops += 2.0 * (double)L * Rr * b * rmax;
        TtmJob fj;
        std::memset(&fj, 0, sizeof(fj));
        fj.X = op(B_Q, h.q_off[n] * 8);
        fj.x_type = T_F64;
        fj.P = op(B_WS, h.P32[n]);
        fj.Y = op(B_OUT, h.out_fac_off[n] * 8);
        fj.y_type = T_F64;
        fj.L = (int64_t)h.n[n];
        fj.Rr = 1;
        fj.b = b;
        fj.rmax = rmax;
        fj.tiles = ttm_rows_tiles((int64_t)h.n[n]);
        fj.tile_begin = (int)fac_tiles;
        fac_tiles += fj.tiles;
        fac2.push_back(fj);
        fac_flops += 2.0 * (double)h.n[n] * b * rmax;
        continue;
      }
      SimtJob t;
      std::memset(&t, 0, sizeof(t));
      t.batch = 1;
      t.alpha = 1.0f;
      if (L == 1) {
        t.M = rmax; t.N = (int)Rr; t.K = b; t.K1 = b;
        t.A = op(B_WS, h.P32[n]); t.a_type = T_F32; t.a_m = b; t.a_k0 = 1;
        t.B = X; t.b_type = xt; t.b_n = b; t.b_k0 = 1;
        t.c_m = 1; t.c_n = rmax;
      } else {
        t.M = (int)L; t.N = rmax; t.K = b; t.K1 = b; t.batch = (int)Rr;
        t.A = X; t.a_type = xt; t.a_m = 1; t.a_k0 = L; t.a_b = L * b;
        t.B = op(B_WS, h.P32[n]); t.b_type = T_F32; t.b_n = b; t.b_k0 = 1;
        t.c_m = 1; t.c_n = L; t.c_b = L * rmax;
      }
      if (n == d - 1) {
        t.has_c64 = 1;
        t.c64 = op(B_OUT, h.out_core_off * 8);
      } else {
        t.has_c32 = 1;
        t.c32 = op(B_WS, h.Hp[n & 1]);
      }
      ttm.push_back(t);
      SimtJob f;
      std::memset(&f, 0, sizeof(f));
      f.batch = 1;
      f.alpha = 1.0f;
      f.M = (int)h.n[n]; f.N = rmax; f.K = b; f.K1 = b;
      f.A = op(B_Q, h.q_off[n] * 8); f.a_type = T_F64; f.a_m = 1; f.a_k0 = h.n[n];
      f.B = op(B_WS, h.P32[n]); f.b_type = T_F32; f.b_n = b; f.b_k0 = 1;
      f.has_c64 = 1;
      f.c64 = op(B_OUT, h.out_fac_off[n] * 8);
      f.c_m = 1;
      f.c_n = h.n[n];
      fac.push_back(f);
    }
    char nm[32];
    for (size_t lvl = 0; lvl < tsqr.size(); ++lvl) {
      std::snprintf(nm, sizeof(nm), "a9:tsqr%d.%d[f32]", n, (int)lvl);
      plan->push(plan->st_recompress, S_TSQR, tsqr[lvl], (int64_t)tsqr[lvl].size(), nm, lvl == 0 ? qflops : 0.0,
                 0.0);
    }
    std::snprintf(nm, sizeof(nm), "a9:svd%d[f32]", n);
    plan->push(plan->st_recompress, S_SVD32, svds, (int64_t)svds.size(), nm);
    std::snprintf(nm, sizeof(nm), "a9:ttm%d[f32]", n);
    plan->push_simt(plan->st_recompress, ttm, nm);
    plan->push(plan->st_recompress, S_TTM, ttm2, ttm_tiles, nm, ttm_flops, 0.0);
    std::snprintf(nm, sizeof(nm), "a9:factor%d[f32]", n);
    plan->push_simt(plan->st_recompress, fac, nm);
    plan->push(plan->st_recompress, S_TTM, fac2, fac_tiles, nm, fac_flops, 0.0);
  }
}

// Backward of the core projection for order-3 problems in float64 (stop-gradient through Q).
// With Hbar (b0 x b1 x b2) and A_n = Q_n^T Ucat_n:
//   Z0 = Hbar x_1 A_0cat^T (R0 x b1 x b2), Z2 = Hbar x_3 A_2cat^T (b0 x b1 x R2)   [all terms]
//   per term k (rank offsets o_n):  Z01 = Z0_k x_2 A_k1^T,  dG_k = alpha_k Z01 x_3 A_k2^T,
//   B_k2 = alpha_k (Z01)_(3) G_k,(3)^T,  W1 = Z0_k x_3 A_k2^T,  B_k1 = alpha_k (W1)_(2) G_k,(2)^T,
//   W0 = Z2_k x_2 A_k1^T,  B_k0 = alpha_k (W0)_(1) G_k,(1)^T;   dUcat_n = Q_n Bcat_n.
static void build_backward3(tks_plan* plan) {
  GemmList big, step1, step2, du;
  for (auto& h : plan->probs) {
    const int b0 = h.b[0], b1 = h.b[1], b2 = h.b[2];
    const int R0 = h.R[0], R2 = h.R[2];
    // Z0[i + R0 J] = sum_a A_0[a + b0 i] Hbar[a + b0 J]
    big.add(gemm(R0, b1 * b2, b0, op(B_WS, h.A[0]), b0, 1, op(B_HBAR, h.h_off * 8), b0, 1, op(B_WS, h.bZ0), 1, R0));
    // Z2[J01 + b0 b1 i] = sum_a Hbar[J01 + b0 b1 a] A_2[a + b2 i]
    big.add(gemm(b0 * b1, R2, b2, op(B_HBAR, h.h_off * 8), 1, (int64_t)b0 * b1, op(B_WS, h.A[2]), b2, 1,
                 op(B_WS, h.bZ2), 1, (int64_t)b0 * b1));
    for (int k = 0; k < h.K; ++k) {
      const int* r = &h.ranks[(size_t)k * 3];
      const int o0 = h.roff[(size_t)k * 3], o1 = h.roff[(size_t)k * 3 + 1], o2 = h.roff[(size_t)k * 3 + 2];
      const double al = h.alpha[k];
      const Operand Z0k = op(B_WS, h.bZ0 + (size_t)o0 * 8);
      const Operand Z2k = op(B_WS, h.bZ2 + (size_t)b0 * b1 * o2 * 8);
      const Operand A1k = op(B_WS, h.A[1] + (size_t)b1 * o1 * 8);
      const Operand A2k = op(B_WS, h.A[2] + (size_t)b2 * o2 * 8);
      const Operand Gk = op_abs(h.cores, (size_t)h.core_off[k] * 8);
      const Operand Z01 = op(B_WS, h.bterm[3 * k]), W1 = op(B_WS, h.bterm[3 * k + 1]);
      const Operand W0 = op(B_WS, h.bterm[3 * k + 2]);
      // Z01[i0 + r0 i1 + r0 r1 j2] = sum_j1 Z0k[i0 + R0 j1 + R0 b1 j2] A_1[j1 + b1 (o1 + i1)]
      GemmJob g = gemm(r[0], r[1], b1, Z0k, 1, R0, A1k, b1, 1, Z01, 1, r[0]);
      g.batch = b2;
      g.a_b = (int64_t)R0 * b1;
      g.c_b = (int64_t)r[0] * r[1];
      step1.add(g);
      // W1[i0 + r0 j1 + r0 b1 i2] = sum_j2 Z0k[i0 + R0 j1 + R0 b1 j2] A_2[j2 + b2 (o2 + i2)]
      g = gemm(r[0], r[2], b2, Z0k, 1, (int64_t)R0 * b1, A2k, b2, 1, W1, 1, (int64_t)r[0] * b1);
      g.batch = b1;
      g.a_b = R0;
      g.c_b = r[0];
      step1.add(g);
      // W0[j0 + b0 i1 + b0 r1 i2] = sum_j1 Z2k[j0 + b0 j1 + b0 b1 i2] A_1[j1 + b1 (o1 + i1)]
      g = gemm(b0, r[1], b1, Z2k, 1, b0, A1k, b1, 1, W0, 1, b0);
      g.batch = r[2];
      g.a_b = (int64_t)b0 * b1;
      g.c_b = (int64_t)b0 * r[1];
      step1.add(g);
      // dG_k[J + r0 r1 i2] = alpha sum_j2 Z01[J + r0 r1 j2] A_2[j2 + b2 (o2 + i2)]
      step2.add(gemm(r[0] * r[1], r[2], b2, Z01, 1, (int64_t)r[0] * r[1], A2k, b2, 1,
                     op(B_DCORE, (size_t)(h.gcore_off + h.core_off[k]) * 8), 1, (int64_t)r[0] * r[1], al));
      // B_k2[j2 + b2 (o2 + i2)] = alpha sum_J Z01[J + r0 r1 j2] G[J + r0 r1 i2]
      step2.add(gemm(b2, r[2], r[0] * r[1], Z01, (int64_t)r[0] * r[1], 1, Gk, (int64_t)r[0] * r[1], 1,
                     op(B_WS, h.bB[2] + (size_t)b2 * o2 * 8), 1, b2, al));
      // B_k1[j1 + b1 (o1 + i1)] = alpha sum_{i0, i2} W1[i0 + r0 j1 + r0 b1 i2] G[i0 + r0 i1 + r0 r1 i2]
      g = gemm(b1, r[1], r[0] * r[2], W1, r[0], 1, Gk, r[0], 1, op(B_WS, h.bB[1] + (size_t)b1 * o1 * 8), 1, b1, al);
      g.K1 = r[0];
      g.a_k1 = (int64_t)r[0] * b1;
      g.b_k1 = (int64_t)r[0] * r[1];
      step2.add(g);
      // B_k0[j0 + b0 (o0 + i0)] = alpha sum_{i1, i2} W0[j0 + b0 (i1 + r1 i2)] G[i0 + r0 (i1 + r1 i2)]
      step2.add(gemm(b0, r[0], r[1] * r[2], W0, 1, b0, Gk, 1, r[0], op(B_WS, h.bB[0] + (size_t)b0 * o0 * 8), 1, b0,
                     al));
    }
    for (int n = 0; n < 3; ++n)
      // dUcat_n[i + n col] = sum_a Q[i + n a] Bcat_n[a + b col]
      du.add(gemm((int)h.n[n], h.R[n], h.b[n], op(B_Q, h.q_off[n] * 8), 1, h.n[n], op(B_WS, h.bB[n]), h.b[n], 1,
                  op(B_DFAC, (size_t)h.gfac_off[n] * 8), 1, h.n[n]));
  }
  plan->push_gemm(plan->st_backward, big, "bwd:Z=Hbar.Acat");
  plan->push_gemm(plan->st_backward, step1, "bwd:per-term1");
  plan->push_gemm(plan->st_backward, step2, "bwd:per-term2");
  plan->push_gemm(plan->st_backward, du, "bwd:dU=Q.B");
}

// The same backward for mixed-precision plans (order 3): the contractions over a basis index with a
// large partner dimension run on the tensor cores as bf16 plane products (hi/mid/lo splits of float64
// and float32 operands, six products up to second order, float32 accumulation in TMEM), the small
// per-term ones in float32 on the CUDA cores:
//   [tc]   A_n^T = Ucat_n^T Q_n (float32, and A_n as planes with the basis index fastest)
//   [tc]   Z0 = Hbar x_1 A_0cat^T,  Z2^T = (Hbar x_3 A_2cat^T)^T
//   [f32]  Z01, W1, W0, then dG_k (float64 out) and B_kn (written as planes of Bcat_n)
//   [tc]   dUcat_n^T = Bcat_n^T Q_n^T (float64 out)
static void simt_set(SimtJob& j, int M, int N, int K, Operand A, int32_t at, int64_t a_m, int64_t a_k0, Operand B,
                     int32_t bt, int64_t b_n, int64_t b_k0, int64_t c_m, int64_t c_n, float alpha) {
  std::memset(&j, 0, sizeof(j));
  j.M = M; j.N = N; j.K = K; j.K1 = K; j.batch = 1;
  j.A = A; j.a_type = at; j.a_m = a_m; j.a_k0 = a_k0;
  j.B = B; j.b_type = bt; j.b_n = b_n; j.b_k0 = b_k0;
  j.c_m = c_m; j.c_n = c_n;
  j.alpha = alpha;
}

static void build_backward3_mixed(tks_plan* plan) {
  std::vector<SplitJob> sp;
  int64_t sp_total = 0;
  std::vector<TcJob> tcA, tcZ, tcU;
  std::vector<SimtJob> step1, step2;
  auto split = [&](Operand src, const size_t* dst, int64_t rows, int64_t cols, int64_t ld_src, int64_t ld_dst,
                   int trans) {
    SplitJob sj;
    std::memset(&sj, 0, sizeof(sj));
    sj.src = src;
    for (int t = 0; t < 3; ++t) sj.dst[t] = op(B_WS, dst[t]);
    sj.rows = rows;
    sj.cols = cols;
    sj.ld_src = ld_src;
    sj.ld_dst = ld_dst;
    sj.trans = trans;
    sj.count = rows * cols;
    sj.begin = 0;
    sj.tile_begin = (int32_t)sp_total;
    sp_total += (sj.count + kSplitTile - 1) / kSplitTile;
    sp.push_back(sj);
  };
  auto tc6 = [](TcJob& j) {
    const uint8_t pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
    j.na = j.nb = 3;
    j.npairs = 6;
    for (int t = 0; t < 6; ++t) {
      j.pa[t] = pa[t];
      j.pb[t] = pb[t];
    }
  };
  for (auto& h : plan->probs) {
    const int b0 = h.b[0], b1 = h.b[1], b2 = h.b[2];
    const int R0 = h.R[0], R2 = h.R[2];
    const Operand Hbar = op(B_HBAR, h.h_off * 8);
    // planes of Q_n (row i fastest, for A_n^T) and of Q_n^T (basis index fastest, for dU), of Hbar
    // with the mode-1 index fastest (Z0) and with the mode-3 index fastest (Z2)
    for (int n = 0; n < 3; ++n) {
      const int64_t nn = h.n[n];
      split(op(B_Q, h.q_off[n] * 8), h.Qp[n], nn, h.b[n], nn, nn, 0);
      split(op(B_Q, h.q_off[n] * 8), h.bQT[n], nn, h.b[n], nn, h.ldb[n], 1);
    }
    split(Hbar, h.bHA, b0, (int64_t)b1 * b2, b0, h.ldb[0], 0);
    split(Hbar, h.bHC, (int64_t)b0 * b1, b2, (int64_t)b0 * b1, h.ldb[2], 1);
    // A_n^T = Ucat_n^T Q_n: exact bf16 factors times the three planes of Q_n
    for (int n = 0; n < 3; ++n) {
      const int64_t nn = h.n[n];
      TcJob j;
      std::memset(&j, 0, sizeof(j));
      j.M = h.R[n]; j.N = h.b[n]; j.K = (int)nn;
      j.epi.alpha = 1.0f;
      j.na = 1; j.nb = 3; j.npairs = 3;
      j.mapA[0] = plan->map_of(B_ABS, reinterpret_cast<uintptr_t>(h.factors[n]), nn, h.R[n], nn, 128);
      for (int t = 0; t < 3; ++t) {
        j.mapB[t] = plan->map_of(B_WS, h.Qp[n][t], nn, h.b[n], nn, 64);
        j.pa[t] = 0;
        j.pb[t] = (uint8_t)t;
      }
      j.epi.has_f32 = 1;
      j.epi.f32 = op(B_WS, h.AT32[n]);
      j.epi.f32_m = 1;
      j.epi.f32_n = h.R[n];
      j.epi.nbf = 3;
      for (int t = 0; t < 3; ++t) j.epi.bf[t] = op(B_WS, h.bAp[n][t]);
      j.epi.bf_m = h.ldb[n];
      j.epi.bf_n = 1;
      tcA.push_back(j);
    }
    // Z0[i + R0 J] = sum_a A_0[a, i] Hbar[a + b0 J]   (M = R0, N = b1 b2, K = b0)
    {
      TcJob j;
      std::memset(&j, 0, sizeof(j));
      j.M = R0; j.N = b1 * b2; j.K = b0;
      j.epi.alpha = 1.0f;
      tc6(j);
      for (int t = 0; t < 3; ++t) {
        j.mapA[t] = plan->map_of(B_WS, h.bAp[0][t], b0, R0, h.ldb[0], 128);
        j.mapB[t] = plan->map_of(B_WS, h.bHA[t], b0, (uint64_t)b1 * b2, h.ldb[0], 64);
      }
      j.epi.has_f32 = 1;
      j.epi.f32 = op(B_WS, h.bZ0);
      j.epi.f32_m = 1;
      j.epi.f32_n = R0;
      tcZ.push_back(j);
    }
    // Z2[J01 + b0 b1 i] = sum_a Hbar[J01 + b0 b1 a] A_2[a, i]   (as Z2^T: M = R2, N = b0 b1, K = b2)
    {
      TcJob j;
      std::memset(&j, 0, sizeof(j));
      j.M = R2; j.N = b0 * b1; j.K = b2;
      j.epi.alpha = 1.0f;
      tc6(j);
      for (int t = 0; t < 3; ++t) {
        j.mapA[t] = plan->map_of(B_WS, h.bAp[2][t], b2, R2, h.ldb[2], 128);
        j.mapB[t] = plan->map_of(B_WS, h.bHC[t], b2, (uint64_t)b0 * b1, h.ldb[2], 64);
      }
      j.epi.has_f32 = 1;
      j.epi.f32 = op(B_WS, h.bZ2);
      j.epi.f32_m = (int64_t)b0 * b1;
      j.epi.f32_n = 1;
      tcZ.push_back(j);
    }
    // per term (rank offsets o_n); A_n[a, r] = AT32_n[r + R_n a]
    for (int k = 0; k < h.K; ++k) {
      const int* r = &h.ranks[(size_t)k * 3];
      const int o0 = h.roff[(size_t)k * 3], o1 = h.roff[(size_t)k * 3 + 1], o2 = h.roff[(size_t)k * 3 + 2];
      const float al = (float)h.alpha[k];
      const Operand Z0k = op(B_WS, h.bZ0 + (size_t)o0 * 4);
      const Operand Z2k = op(B_WS, h.bZ2 + (size_t)b0 * b1 * o2 * 4);
      const Operand A0k = op(B_WS, h.AT32[0] + (size_t)o0 * 4);
      const Operand A1k = op(B_WS, h.AT32[1] + (size_t)o1 * 4);
      const Operand A2k = op(B_WS, h.AT32[2] + (size_t)o2 * 4);
      const int64_t R1 = h.R[1];
      const Operand Gk = op_abs(h.cores, (size_t)h.core_off[k] * 2);
      const Operand Z01 = op(B_WS, h.bterm[3 * k]), W1 = op(B_WS, h.bterm[3 * k + 1]);
      const Operand W0 = op(B_WS, h.bterm[3 * k + 2]);
      SimtJob g;
      // Z01[i0 + r0 i1 + r0 r1 j2] = sum_j1 Z0k[i0 + R0 j1 + R0 b1 j2] A_1[j1, o1 + i1]
      simt_set(g, r[0], r[1], b1, Z0k, T_F32, 1, R0, A1k, T_F32, 1, R1, 1, r[0], 1.0f);
      g.batch = b2; g.a_b = (int64_t)R0 * b1; g.c_b = (int64_t)r[0] * r[1];
      g.has_c32 = 1; g.c32 = Z01;
      step1.push_back(g);
      // W1[i0 + r0 j1 + r0 b1 i2] = sum_j2 Z0k[i0 + R0 j1 + R0 b1 j2] A_2[j2, o2 + i2]
      simt_set(g, r[0], r[2], b2, Z0k, T_F32, 1, (int64_t)R0 * b1, A2k, T_F32, 1, R2, 1, (int64_t)r[0] * b1, 1.0f);
      g.batch = b1; g.a_b = R0; g.c_b = r[0];
      g.has_c32 = 1; g.c32 = W1;
      step1.push_back(g);
      // W0[j0 + b0 i1 + b0 r1 i2] = sum_j1 Z2k[j0 + b0 j1 + b0 b1 i2] A_1[j1, o1 + i1]
      simt_set(g, b0, r[1], b1, Z2k, T_F32, 1, b0, A1k, T_F32, 1, R1, 1, b0, 1.0f);
      g.batch = r[2]; g.a_b = (int64_t)b0 * b1; g.c_b = (int64_t)b0 * r[1];
      g.has_c32 = 1; g.c32 = W0;
      step1.push_back(g);
      // dG_k[J + r0 r1 i2] = alpha sum_j2 Z01[J + r0 r1 j2] A_2[j2, o2 + i2]
      simt_set(g, r[0] * r[1], r[2], b2, Z01, T_F32, 1, (int64_t)r[0] * r[1], A2k, T_F32, 1, R2, 1,
               (int64_t)r[0] * r[1], al);
      g.has_c64 = 1; g.c64 = op(B_DCORE, (size_t)(h.gcore_off + h.core_off[k]) * 8);
      step2.push_back(g);
      // Bcat_2[j2, o2 + i2] = alpha sum_J Z01[J + r0 r1 j2] G[J + r0 r1 i2]
      simt_set(g, b2, r[2], r[0] * r[1], Z01, T_F32, (int64_t)r[0] * r[1], 1, Gk, T_BF16, (int64_t)r[0] * r[1], 1, 1,
               h.ldb[2], al);
      g.nbf = 3;
      for (int t = 0; t < 3; ++t) g.cb[t] = op(B_WS, h.bBp[2][t] + (size_t)h.ldb[2] * o2 * 2);
      step2.push_back(g);
      // Bcat_1[j1, o1 + i1] = alpha sum_{i0, i2} W1[i0 + r0 j1 + r0 b1 i2] G[i0 + r0 i1 + r0 r1 i2]
      simt_set(g, b1, r[1], r[0] * r[2], W1, T_F32, r[0], 1, Gk, T_BF16, r[0], 1, 1, h.ldb[1], al);
      g.K1 = r[0];
      g.a_k1 = (int64_t)r[0] * b1;
      g.b_k1 = (int64_t)r[0] * r[1];
      g.nbf = 3;
      for (int t = 0; t < 3; ++t) g.cb[t] = op(B_WS, h.bBp[1][t] + (size_t)h.ldb[1] * o1 * 2);
      step2.push_back(g);
      // Bcat_0[j0, o0 + i0] = alpha sum_{i1, i2} W0[j0 + b0 (i1 + r1 i2)] G[i0 + r0 (i1 + r1 i2)]
      simt_set(g, b0, r[0], r[1] * r[2], W0, T_F32, 1, b0, Gk, T_BF16, 1, r[0], 1, h.ldb[0], al);
      g.nbf = 3;
      for (int t = 0; t < 3; ++t) g.cb[t] = op(B_WS, h.bBp[0][t] + (size_t)h.ldb[0] * o0 * 2);
      step2.push_back(g);
      (void)A0k;
    }
    // dUcat_n^T = Bcat_n^T Q_n^T: dfac[i + n col] (M = R_n, N = n_n, K = b_n)
    for (int n = 0; n < 3; ++n) {
      const int64_t nn = h.n[n];
      TcJob j;
      std::memset(&j, 0, sizeof(j));
      j.M = h.R[n]; j.N = (int)nn; j.K = h.b[n];
      j.epi.alpha = 1.0f;
      tc6(j);
      for (int t = 0; t < 3; ++t) {
        j.mapA[t] = plan->map_of(B_WS, h.bBp[n][t], h.b[n], h.R[n], h.ldb[n], 128);
        j.mapB[t] = plan->map_of(B_WS, h.bQT[n][t], h.b[n], nn, h.ldb[n], 64);
      }
      j.epi.has_f64 = 1;
      j.epi.f64 = op(B_DFAC, (size_t)h.gfac_off[n] * 8);
      j.epi.f64_m = nn;
      j.epi.f64_n = 1;
      tcU.push_back(j);
    }
  }
  plan->push(plan->st_backward, S_SPLIT, sp, sp_total, "bwd:Q,Hbar->planes", 0.0, 14.0 * kSplitTile * sp_total);
  plan->push_tc(plan->st_backward, tcA, "bwd:AT=UcatT.Q[tc]");
  plan->push_tc(plan->st_backward, tcZ, "bwd:Z=Hbar.Acat[tc]");
  plan->push_simt(plan->st_backward, step1, "bwd:per-term1[f32]");
  plan->push_simt(plan->st_backward, step2, "bwd:per-term2[f32]");
  plan->push_tc(plan->st_backward, tcU, "bwd:dUT=BT.QT[tc]");
}

}  // namespace

// ST-HOSVD of H in float64 (TKS_FP64 and TKS_MIXED; Alg. 2 phase 2, modes 1..d in order): per mode,
// TSQR of H_(n)^T (rows = the other modes, two-level index) in float64, one-sided Jacobi SVD of its
// b x b triangular factor (right singular vectors = left singular vectors of H_(n)), rank rule, then
// H <- H x_n P_n^T and U~_n = Q_n P_n as float64 GEMMs; problems [lane_p0, lane_p1).
static void build_hosvd_f64(tks_plan* plan) {
  for (int n = 0; n < plan->dmax; ++n) {
    std::vector<std::vector<TsqrJob>> tsqr;
    std::vector<SvdJob> svds;
    double svd_flops = 0.0;
    std::vector<TtmJob> ttm, fac;
    std::vector<OzSliceJob> oz_slices;
    std::vector<OzGemmJob> oz_gemms;
    int64_t oz_slice_total = 0, oz_gemm_total = 0;
    // TKS_MIXED: the mode products run float64-accurate on the tensor cores (Ozaki scheme)
    const bool emulate = plan->params.precision == TKS_MIXED;
    int64_t ttm_tiles = 0, fac_tiles = 0;
    double qflops = 0.0, ttm_flops = 0.0, fac_flops = 0.0;
    // TKS_MIXED with b <= 64: the triangular factor by shifted CholeskyQR3 with float64-accurate Gram
    // matrices and products on the tensor cores (the Householder TSQR below runs only where it fails)
    CqLists cq;
    for (int p = plan->lane_p0; p < plan->lane_p1; ++p) {
      auto& h = plan->probs[p];
      const int d = h.d;
      if (n >= d) continue;
      int64_t L = 1, Rr = 1;
      for (int j = 0; j < n; ++j) L *= h.rmax[j];
      for (int j = n + 1; j < d; ++j) Rr *= h.b[j];
      const int b = h.b[n], rmax = h.rmax[n];
      const Operand X = (n == 0) ? op(B_H, h.h_off * 8) : op(B_WS, h.Hp[(n - 1) & 1]);
      const bool cholqr = emulate && b <= 64 && plan->params.hosvd_r != 2;
      Operand gate{B_NONE, 0, 0};
      if (cholqr) {
        const CqBuffers B{{h.cqX[0], h.cqX[1]}, h.cqCol, h.cqColE, h.cqG, h.cqRinv, h.cqRacc, h.cqFlag,
                          h.ozA, h.ozEA, h.ozB, h.ozEB, h.cqPart, h.cqCol2, h.cqColE2};
        gate = cq.add(plan, X, L * Rr, L, b, B, op(B_WS, h.R64), Operand{B_NONE, 0, 0},
                      plan->params.hosvd_r == 3 ? 2 : 3);
      }
      // TSQR of H_(n)^T: element (l + L rr, c) at l + L c + L b rr.  Level 0 factors blocks of dense
      // rows; every later level factors groups of the previous level's b x b triangular factors,
      // each group read with its factors' rows interleaved (row f + k r of a group of k is row r of
      // factor f), so that column j of the group is zero below row k (j + 1) and the kernel skips
      // those rows.  The last level writes R64.
      {
        const int64_t rows0 = L * Rr;
        qflops += 2.0 * (double)rows0 * b * b;
        const int brows_max = tsqr64_block_rows(plan->bmax);
        const int nblk0 = std::max(1, ceil_div(rows0, brows_max));
        const int brows0 = ceil_div(rows0, nblk0);
        int nfac = nblk0;               // factors written by the level just planned
        int64_t ld_prev = 0;
        Operand prev;
        for (int lvl = 0;; ++lvl) {
          const int kf_max = std::max(2, brows_max / b);
          const int nblk = lvl == 0 ? nblk0 : std::max(1, ceil_div(nfac, kf_max));
          if (lvl > 0 && nblk > 1 && nblk >= nfac) {   // groups of at least two factors always shrink
            plan->build_error = "TSQR levels do not shrink";
            return;
          }
          const bool final_level = (nblk == 1);
          const Operand dst = final_level ? op(B_WS, h.R64) : op(B_WS, h.stk64[lvl & 1]);
          const int64_t dst_ld = final_level ? b : (int64_t)nblk * b;
          if ((int)tsqr.size() <= lvl) tsqr.resize(lvl + 1);
          for (int i = 0; i < nblk; ++i) {
            TsqrJob t;
            std::memset(&t, 0, sizeof(t));
            t.gate = gate;
            t.src_type = T_F64;
            t.cols = b;
            t.dst = dst;
            t.dst_row0 = (int64_t)i * b;
            t.dst_ld = dst_ld;
            if (lvl == 0) {
              t.src = X;
              t.row_begin = (int64_t)i * brows0;
              t.rows = (int)std::min<int64_t>(brows0, rows0 - t.row_begin);
              t.L0 = L;
              t.s0 = 1;
              t.s1 = L * b;
              t.sc = L;
            } else {
              // factors [f0, f1) of the previous level, spread evenly over the groups
              const int f0 = (int)((int64_t)i * nfac / nblk), f1 = (int)((int64_t)(i + 1) * nfac / nblk);
              t.src = prev;
              t.src.off += (int64_t)f0 * b * 8;
              t.row_begin = 0;
              t.rows = (f1 - f0) * b;
              t.L0 = f1 - f0;
              t.s0 = b;
              t.s1 = 1;
              t.sc = ld_prev;
              t.tri = f1 - f0;
            }
            tsqr[lvl].push_back(t);
          }
          if (final_level) break;
          prev = dst;
          ld_prev = dst_ld;
          nfac = nblk;
        }
      }
      SvdJob sj;
      std::memset(&sj, 0, sizeof(sj));
      sj.R = op(B_WS, h.R64);
      sj.P = op(B_WS, h.P[n]);
      sj.sv = op(B_WS, h.ev[n]);
      sj.theta = op(B_WS, h.theta);
      sj.rank = op(B_RANKS, (size_t)(p * TKS_MAX_ORDER + n) * 4);
      sj.b = b;
      sj.rmax = rmax;
      sj.first_mode = (n == 0);
      sj.mode = n;
      sj.err = op(B_WS, h.errw);
      sj.order = d;
      sj.tol = plan->params.trunc_tol;
      svds.push_back(sj);
      // algorithmic count of an SVD giving the singular values and left vectors of a b x b matrix:
      // Golub and Van Loan's R-SVD, 4 m^2 n + 22 n^3 with m = n = b (Jacobi executes its own count)
      svd_flops += 26.0 * (double)b * b * b;
      // H x_n P_n^T (fibres (l, rr) of H_(n)) and U~_n = Q_n P_n (fibres = rows of Q_n)
      TtmJob tj;
      std::memset(&tj, 0, sizeof(tj));
      tj.X = X;
      tj.x_type = T_F64;
      tj.P = op(B_WS, h.P[n]);
      tj.Y = (n == d - 1) ? op(B_OUT, h.out_core_off * 8) : op(B_WS, h.Hp[n & 1]);
      tj.y_type = T_F64;
      tj.L = L;
      tj.Rr = Rr;
      tj.b = b;
      tj.rmax = rmax;
      tj.tiles = ttm64_tiles(L * Rr);
      tj.tile_begin = (int)ttm_tiles;
      ttm_tiles += tj.tiles;
      ttm.push_back(tj);
      ttm_flops += 2.0 * (double)L * Rr * b * rmax;
      TtmJob fj = tj;
      fj.X = op(B_Q, h.q_off[n] * 8);
      fj.Y = op(B_OUT, h.out_fac_off[n] * 8);
      fj.L = (int64_t)h.n[n];
      fj.Rr = 1;
      fj.tiles = ttm64_tiles((int64_t)h.n[n]);
      fj.tile_begin = (int)fac_tiles;
      fac_tiles += fj.tiles;
      fac.push_back(fj);
      fac_flops += 2.0 * (double)h.n[n] * b * rmax;
      if (emulate) {
        // the same two products, float64-accurate on the tensor cores: digit planes of the fibres
        // of H_(n), of the rows of Q_n and of the columns of P_n, then 128 x 64 tiles of Y
        const int ldk = b <= 64 ? 64 : 128;
        auto slice = [&](Operand src, size_t planes, size_t expo, int64_t rows, int64_t Ls,
                         Operand kexp = Operand{B_NONE, 0, 0}) {
          OzSliceJob sj2;
          std::memset(&sj2, 0, sizeof(sj2));
          sj2.kexp = kexp;
          sj2.src = src;
          sj2.planes = op(B_WS, planes);
          sj2.expo = op(B_WS, expo);
          sj2.rows = rows;
          sj2.L = Ls;
          sj2.rows_pad = (rows + 7) / 8 * 8;
          sj2.K = b;
          sj2.ld = ldk;
          sj2.tiles = oz_slice_tiles(rows);
          sj2.tile_begin = (int)oz_slice_total;
          oz_slice_total += sj2.tiles;
          oz_slices.push_back(sj2);
          return sj2;
        };
        // with CholeskyQR, pass 1 already cut H_(n)^T into digits against its column exponents (the
        // column planes in cqCol): the mode product reads them MN-major, with those exponents folded
        // into the rows of P_n (no row exponents of X); Q_n P_n takes P_n's own digits
        OzSliceJob sx;
        if (cholqr) {
          std::memset(&sx, 0, sizeof(sx));
          sx.planes = op(B_WS, h.cqCol);
          sx.expo = Operand{B_NONE, 0, 0};
          sx.rows = L * Rr;
          sx.rows_pad = (sx.rows + 7) / 8 * 8;
        } else {
          sx = slice(X, h.ozA, h.ozEA, L * Rr, L);
        }
        const OzSliceJob sp = cholqr ? slice(op(B_WS, h.P[n]), h.ozB, h.ozEB, rmax, 1, op(B_WS, h.cqColE))
                                     : slice(op(B_WS, h.P[n]), h.ozB, h.ozEB, rmax, 1);
        const OzSliceJob spq = cholqr ? slice(op(B_WS, h.P[n]), h.ozB2, h.ozEB2, rmax, 1) : sp;
        const OzSliceJob sq = slice(op(B_Q, h.q_off[n] * 8), h.ozQ, h.ozEQ, (int64_t)h.n[n], (int64_t)h.n[n]);
        auto gemm_job = [&](const OzSliceJob& a, const OzSliceJob& sp, Operand Yop, int64_t Ly, bool a_mn) {
          OzGemmJob g;
          std::memset(&g, 0, sizeof(g));
          g.M = (int)a.rows;
          g.N = rmax;
          g.K = b;
          g.tiles_m = ceil_div(g.M, 128);
          g.tiles_n = ceil_div(g.N, 64);
          g.tile_begin = (int)oz_gemm_total;
          oz_gemm_total += (int64_t)g.tiles_m * g.tiles_n;
          for (int sl = 0; sl < kOzSlices; ++sl) {
            // column planes (a_mn): 64 rows of rows_pad digits per plane, boxes of 64 rows x 64 k
            g.mapA[sl] = a_mn ? plan->map_of(B_WS, a.planes.off + (size_t)sl * 64 * a.rows_pad * 2, a.rows, b,
                                             a.rows_pad, 64)
                              : plan->map_of(B_WS, a.planes.off + (size_t)sl * a.rows_pad * ldk * 2, b, a.rows, ldk, 128);
            g.mapB[sl] = plan->map_of(B_WS, sp.planes.off + (size_t)sl * sp.rows_pad * ldk * 2, b, rmax, ldk, 64);
          }
          g.a_mn = a_mn ? 1 : 0;
          g.expA = a.expo;
          g.expB = sp.expo;
          g.Y = Yop;
          g.L = Ly;
          g.rmax = rmax;
          oz_gemms.push_back(g);
        };
        gemm_job(sx, sp, tj.Y, L, cholqr);
        gemm_job(sq, spq, fj.Y, (int64_t)h.n[n], false);
      }
    }
    char nm[32];
    {
      char tag[24];
      std::snprintf(tag, sizeof(tag), "a9:cq%d", n);
      cq.push(plan, plan->st_recompress, tag);
    }
    // the Householder TSQR: every problem on the TKS_FP64 path and those with b > 64; on the
    // CholeskyQR3 path it is gated per problem and runs only where a Cholesky step broke down
    const bool any_tsqr_work = cq.gram[0].empty();
    for (size_t lvl = 0; lvl < tsqr.size(); ++lvl) {
      std::snprintf(nm, sizeof(nm), "a9:tsqr%d.%d", n, (int)lvl);
      plan->push(plan->st_recompress, S_TSQR64, tsqr[lvl], (int64_t)tsqr[lvl].size(), nm,
                 lvl == 0 && any_tsqr_work ? qflops : 0.0, 0.0);
    }
    std::snprintf(nm, sizeof(nm), "a9:svd%d", n);
    plan->push(plan->st_recompress, S_SVD64, svds, (int64_t)svds.size(), nm, svd_flops, 0.0);
    if (emulate) {
      std::snprintf(nm, sizeof(nm), "a9:slice%d[oz]", n);
      plan->push(plan->st_recompress, S_OZSLICE, oz_slices, oz_slice_total, nm);
      std::snprintf(nm, sizeof(nm), "a9:ttm+factor%d[oz]", n);
      plan->push(plan->st_recompress, S_OZGEMM, oz_gemms, oz_gemm_total, nm, ttm_flops + fac_flops, 0.0);
    } else {
      int max_cols = 1;
      for (const auto& t : ttm) max_cols = std::max(max_cols, t.rmax);
      std::snprintf(nm, sizeof(nm), "a9:ttm%d", n);
      plan->push(plan->st_recompress, S_TTM64, ttm, ttm_tiles, nm, ttm_flops, 0.0);
      if (!ttm.empty()) plan->st_recompress.back().nb_max = max_cols;   // column groups of the kernel
      std::snprintf(nm, sizeof(nm), "a9:factor%d", n);
      plan->push(plan->st_recompress, S_TTM64, fac, fac_tiles, nm, fac_flops, 0.0);
      if (!fac.empty()) plan->st_recompress.back().nb_max = max_cols;
    }
  }
}

extern "C" {

const char* tks_last_error(void) { return g_last_error.c_str(); }

const char* tks_status_string(tks_status s) {
  switch (s) {
    case TKS_OK: return "TKS_OK";
    case TKS_EINVAL: return "TKS_EINVAL";
    case TKS_ENOMEM: return "TKS_ENOMEM";
    case TKS_ECUDA: return "TKS_ECUDA";
    case TKS_ETIMEOUT: return "TKS_ETIMEOUT";
    case TKS_ENONFINITE: return "TKS_ENONFINITE";
    case TKS_ENOCONV: return "TKS_ENOCONV";
    case TKS_EUNSUPPORTED: return "TKS_EUNSUPPORTED";
  }
  return "TKS_UNKNOWN";
}

void tks_plan_destroy(tks_plan* plan) {
  if (!plan) return;
  plan->profile_clear();
  for (cudaStream_t st : plan->lane_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : plan->lane_join) cudaEventDestroy(ev);
  if (plan->lane_fork) cudaEventDestroy(plan->lane_fork);
  if (plan->maps_host) cudaFreeHost(plan->maps_host);
  if (plan->arena_dev) cudaFree(plan->arena_dev);
  delete plan;
}

static tks_status create_plan(tks_plan** out, const tks_problem* problems, int32_t num_problems,
                              const tks_params* params) {
  if (!out) return fail(TKS_EINVAL, "plan output pointer is NULL");
  *out = nullptr;
  if (!problems || !params || num_problems < 1) return fail(TKS_EINVAL, "no problems or params");
  if (num_problems > kMaxProblems) return fail(TKS_EINVAL, "more than 2^20 problems in one plan");
  const tks_params prm = *params;
  if (prm.sketch != TKS_SKETCH_KRP && prm.sketch != TKS_SKETCH_KRON) return fail(TKS_EINVAL, "bad sketch");
  if (!(prm.trunc_tol >= 0.0) || !std::isfinite(prm.trunc_tol)) return fail(TKS_EINVAL, "bad trunc_tol");
  if (prm.omega_lowprec != 0 && prm.omega_lowprec != 1) return fail(TKS_EINVAL, "omega_lowprec must be 0 or 1");
  if (prm.lanes < 0 || prm.lanes > 8) return fail(TKS_EINVAL, "lanes must be 0..8");
  if (prm.autotune != 0 && prm.autotune != 1) return fail(TKS_EINVAL, "autotune must be 0 or 1");
  if (prm.sketch_qr < 0 || prm.sketch_qr > 3) return fail(TKS_EINVAL, "sketch_qr must be 0..3");
  if (prm.hosvd_r < 0 || prm.hosvd_r > 3) return fail(TKS_EINVAL, "hosvd_r must be 0..3");
  if (prm.proj_chunk != 0 && prm.proj_chunk != 8 && prm.proj_chunk != 16)
    return fail(TKS_EINVAL, "proj_chunk must be 0, 8 or 16");
  if (prm.tc_stages != 0 && (prm.tc_stages < 2 || prm.tc_stages > 4)) return fail(TKS_EINVAL, "tc_stages must be 0 or 2..4");
  if (prm.precision == TKS_FP64) {
    if (prm.dtype != TKS_DT_F64) return fail(TKS_EINVAL, "TKS_FP64 needs float64 cores and factors");
  } else if (prm.precision == TKS_MIXED || prm.precision == TKS_MIXED_F32LA) {
    if (prm.dtype != TKS_DT_BF16) return fail(TKS_EINVAL, "the mixed modes need bfloat16 cores and factors");
  } else {
    return fail(TKS_EINVAL, "bad precision");
  }

  auto* plan = new tks_plan();
  plan->params = prm;
  plan->nprob = num_problems;
  plan->probs.resize(num_problems);
  const int kron = prm.sketch == TKS_SKETCH_KRON;
  const bool mixed = prm.precision != TKS_FP64;
  const bool f32la = prm.precision == TKS_MIXED_F32LA;
  for (int p = 0; p < num_problems; ++p) {
    tks_status st = validate_and_size(problems[p], prm, plan->probs[p], p);
    if (st == TKS_OK && mixed) {
      // the tensor-core stages read Ucat_m by TMA: 16-byte aligned rows of n_m bf16
      const auto& h = plan->probs[p];
      for (int m = 0; m < h.d && st == TKS_OK; ++m) {
        if (h.n[m] % 8 != 0)
          st = fail(TKS_EUNSUPPORTED, "problem " + std::to_string(p) + ": TKS_MIXED needs n_m % 8 == 0");
        else if (reinterpret_cast<uintptr_t>(h.factors[m]) % 16 != 0)
          st = fail(TKS_EINVAL, "problem " + std::to_string(p) + ": factor pointer not 16-byte aligned");
      }
    }
    if (st != TKS_OK) {
      delete plan;
      return st;
    }
    count_flops(plan->probs[p], kron);
    plan->flops_low += plan->probs[p].flops_low;
    plan->flops_f64 += plan->probs[p].flops_f64;
    plan->dmax = std::max(plan->dmax, plan->probs[p].d);
    for (int m = 0; m < plan->probs[p].d; ++m) plan->bmax = std::max(plan->bmax, plan->probs[p].b[m]);
  }

  // ---- caller-visible buffer layouts (elements) and workspace (bytes)
  size_t ws = 0;
  auto alloc = [&](size_t bytes) {
    const size_t o = ws;
    ws = align_up(ws + std::max<size_t>(bytes, 1));
    return o;
  };
  for (auto& h : plan->probs) {
    for (int m = 0; m < h.d; ++m) {
      h.omega_off[m] = plan->omega_elems;
      plan->omega_elems += h.n[m] * h.s[m];
      h.y_off[m] = plan->sketch_elems;
      plan->sketch_elems += h.n[m] * h.S[m];
      h.q_off[m] = plan->basis_elems;
      plan->basis_elems += h.n[m] * h.b[m];
    }
    h.h_off = plan->core_elems;
    plan->core_elems += prod(h.b, h.d);
    h.out_core_off = plan->output_elems;
    plan->output_elems += prod(h.rmax, h.d);
    for (int m = 0; m < h.d; ++m) {
      h.out_fac_off[m] = plan->output_elems;
      plan->output_elems += h.n[m] * h.rmax[m];
    }
  }
  for (auto& h : plan->probs) {
    h.gcore_off = plan->grad_core_elems;
    for (int k = 0; k < h.K; ++k) plan->grad_core_elems += prod(&h.ranks[(size_t)k * h.d], h.d);
    for (int m = 0; m < h.d; ++m) {
      h.gfac_off[m] = plan->grad_factor_elems;
      plan->grad_factor_elems += h.n[m] * h.R[m];
    }
  }
  plan->backward_ok = true;
  for (auto& h : plan->probs)
    if (h.d != 3) plan->backward_ok = false;
  plan->ws_omega = alloc(plan->omega_elems * 8);
  plan->ws_Y = alloc(plan->sketch_elems * 8);
  plan->ws_Q = alloc(plan->basis_elems * 8);
  plan->ws_H = alloc(plan->core_elems * 8);
  for (auto& h : plan->probs) h.errw = alloc((1 + TKS_MAX_ORDER) * sizeof(double));
  for (auto& h : plan->probs) {
    const int d = h.d;
    auto r8 = [](int x) { return (x + 7) / 8 * 8; };
    int64_t Pd = 1;
    for (int j = 0; j + 1 < d; ++j) Pd *= h.b[j];
    for (int m = 0; m < d; ++m) {
      h.W[m] = alloc((size_t)h.n[m] * h.S[m] * 8);
      h.tau[m] = alloc((size_t)h.S[m] * 8);
      h.P[m] = alloc((size_t)h.b[m] * h.rmax[m] * 8);
      h.ev[m] = alloc((size_t)h.b[m] * 8);
      if (!mixed) {
        h.M[m] = alloc((size_t)h.R[m] * h.s[m] * 8);
        h.V[m] = alloc((size_t)h.R[m] * h.S[m] * 8);
        h.A[m] = alloc((size_t)h.b[m] * h.R[m] * 8);
      } else {
        h.ldU[m] = h.ldV[m] = h.ldA[m] = r8(h.R[m]);
        h.om_plane[m] = alloc((size_t)h.n[m] * h.s[m] * 2);
        h.M32[m] = alloc((size_t)h.R[m] * h.s[m] * 4);
        for (int t = 0; t < 3; ++t) h.Vp[m][t] = alloc((size_t)h.ldV[m] * h.S[m] * 2);
        for (int t = 0; t < 3; ++t) h.Qp[m][t] = alloc((size_t)h.n[m] * h.b[m] * 2);
        h.AT32[m] = alloc((size_t)h.R[m] * h.b[m] * 4);
        if (prm.precision == TKS_MIXED && h.n[m] >= h.S[m] && h.S[m] <= 64 && prm.sketch_qr != 2) {
          // CholeskyQR3 of Y_n (n_m x S_m): see CqBuffers
          const int64_t rows8 = (h.n[m] + 7) / 8 * 8;
          CqBuffers& B = h.qcq[m];
          B.X[0] = alloc((size_t)h.n[m] * h.S[m] * 8);
          B.X[1] = alloc((size_t)h.n[m] * h.S[m] * 8);
          B.col = alloc((size_t)kOzSlices * 64 * rows8 * 2);
          B.colE = alloc(64 * 4);
          B.G = alloc(64 * 64 * 8);
          B.Rinv = alloc(64 * 64 * 8);
          B.Racc = alloc(64 * 64 * 8);
          B.flag = alloc(4);
          B.rowB = alloc((size_t)kOzSlices * 64 * 64 * 2);
          B.rowBE = alloc(64 * 4);
          B.part = alloc((size_t)ceil_div(h.n[m], 64) * 64 * 4);
          B.col2 = B.col;
          B.colE2 = B.colE;
        }
      }
    }
    if (!mixed) {
      h.T = alloc((size_t)h.R[d - 1] * Pd * 8);
    } else {
      h.fused3 = d == 3 && h.b[1] <= 64 && h.b[2] <= 64;
      if (d == 4 && h.b[2] <= 64 && h.b[3] <= 64) {
        bool fits = true;
        int64_t per_a1 = 0;
        h.g4_off.assign(h.K, 0);
        for (int k = 0; k < h.K; ++k) {
          const int* r = &h.ranks[(size_t)k * d];
          fits = fits && fold4_smem_bytes(r[0], r[1], r[2], h.b[1]) <= 200 * 1024 &&
                 (int64_t)r[0] * r[2] * 4 <= kProj3SliceBytes;   // one float32 slice G'[:, :, i3]
          h.g4_off[k] = per_a1 * h.b[1];
          per_a1 += (int64_t)r[0] * r[2] * r[3];
        }
        h.fused4 = fits;
        if (fits) h.g4 = alloc((size_t)per_a1 * h.b[1] * 4);
      }
      if (!h.fused3 && !h.fused4) {
        // planes of A_d^T and of Tcat for the last-mode tensor-core product
        for (int t = 0; t < 3; ++t) h.ATp[d - 1][t] = alloc((size_t)h.ldA[d - 1] * h.b[d - 1] * 2);
        h.ldT = r8(h.R[d - 1]);
        for (int t = 0; t < 3; ++t) h.Tp[t] = alloc((size_t)h.ldT * Pd * 2);
      }
    }
    h.chain.resize((size_t)2 * h.K);
    for (int k = 0; k < h.K; ++k) {
      const int* r = &h.ranks[(size_t)k * d];
      int64_t mx = 1;
      for (int t = 0; t + 2 < d; ++t) {     // sizes after chain steps 0..d-3
        int64_t sz = 1;
        for (int j = 0; j <= t; ++j) sz *= h.b[j];
        for (int j = t + 1; j < d; ++j) sz *= r[j];
        mx = std::max(mx, sz);
      }
      h.chain[2 * k] = alloc(mx * 8);
      h.chain[2 * k + 1] = alloc(mx * 8);
    }
    int bm = 0;
    for (int m = 0; m < d; ++m) bm = std::max(bm, h.b[m]);
    int64_t Hsz = prod(h.b, d);
    h.theta = alloc(8);
    h.Hp[0] = alloc(Hsz * 8);
    h.Hp[1] = alloc(Hsz * 8);
    if (plan->backward_ok) {
      h.bZ0 = alloc((size_t)h.R[0] * h.b[1] * h.b[2] * 8);
      h.bZ2 = alloc((size_t)h.b[0] * h.b[1] * h.R[2] * 8);
      for (int m = 0; m < 3; ++m) h.bB[m] = alloc((size_t)h.b[m] * h.R[m] * 8);
      h.bterm.resize((size_t)3 * h.K);
      for (int k = 0; k < h.K; ++k) {
        const int* r = &h.ranks[(size_t)k * 3];
        h.bterm[3 * k] = alloc((size_t)r[0] * r[1] * h.b[2] * 8);
        h.bterm[3 * k + 1] = alloc((size_t)r[0] * h.b[1] * r[2] * 8);
        h.bterm[3 * k + 2] = alloc((size_t)h.b[0] * r[1] * r[2] * 8);
      }
      if (mixed) {
        for (int m = 0; m < 3; ++m) {
          h.ldb[m] = (h.b[m] + 7) / 8 * 8;
          for (int t = 0; t < 3; ++t) {
            h.bAp[m][t] = alloc((size_t)h.R[m] * h.ldb[m] * 2);
            h.bBp[m][t] = alloc((size_t)h.R[m] * h.ldb[m] * 2);
            h.bQT[m][t] = alloc((size_t)h.n[m] * h.ldb[m] * 2);
          }
        }
        for (int t = 0; t < 3; ++t) {
          h.bHA[t] = alloc((size_t)h.b[1] * h.b[2] * h.ldb[0] * 2);
          h.bHC[t] = alloc((size_t)h.b[0] * h.b[1] * h.ldb[2] * 2);
        }
      }
    }
    if (!f32la) {
      // float64 TSQR stacks: at most ceil(rows / block) factors of b rows per level
      int64_t stack_rows = 0;
      for (int m = 0; m < d; ++m) {
        const int64_t rows = Hsz / h.b[m];
        stack_rows = std::max<int64_t>(stack_rows, (int64_t)ceil_div(rows, tsqr64_block_rows(plan->bmax)) * h.b[m]);
      }
      h.R64 = alloc((size_t)bm * bm * 8);
      h.stk64[0] = alloc((size_t)stack_rows * bm * 8);
      h.stk64[1] = alloc((size_t)stack_rows * bm * 8);
      if (prm.precision == TKS_MIXED) {
        // digit planes (kOzSlices bf16 planes, rows of 64 or 128 k) and row exponents of the mode
        // products: the fibres of H_(n) (largest mode), the rows of Q_n, the columns of P_n
        const int ldk = bm <= 64 ? 64 : 128;
        int64_t fib = 0, nrow = 0, cols = 0;
        for (int m = 0; m < d; ++m) {
          int64_t L = 1, Rr = 1;
          for (int j = 0; j < m; ++j) L *= h.rmax[j];
          for (int j = m + 1; j < d; ++j) Rr *= h.b[j];
          fib = std::max<int64_t>(fib, (L * Rr + 7) / 8 * 8);
          nrow = std::max<int64_t>(nrow, (h.n[m] + 7) / 8 * 8);
          cols = std::max<int64_t>(cols, (h.rmax[m] + 7) / 8 * 8);
        }
        // with CholeskyQR3 (b <= 64) the b columns of R^-1 also go through the P digit planes
        if (bm <= 64) cols = std::max<int64_t>(cols, (bm + 7) / 8 * 8);
        h.ozA = alloc((size_t)kOzSlices * fib * ldk * 2);
        h.ozQ = alloc((size_t)kOzSlices * nrow * ldk * 2);
        h.ozB = alloc((size_t)kOzSlices * cols * ldk * 2);
        h.ozEA = alloc((size_t)fib * 4);
        h.ozEQ = alloc((size_t)nrow * 4);
        h.ozEB = alloc((size_t)cols * 4);
        // shifted CholeskyQR3 (b <= 64): two X buffers, column digit planes (64 rows of ldP), the Gram
        // matrix, R^-1, the accumulated R, the fallback flag
        if (bm <= 64) {
          const int64_t ldP = fib;   // fib is a multiple of 8 and at least every mode's row count
          h.cqX[0] = alloc((size_t)fib * bm * 8);
          h.cqX[1] = alloc((size_t)fib * bm * 8);
          h.cqCol = alloc((size_t)kOzSlices * 64 * ldP * 2);
          h.cqColE = alloc(64 * 4);
          h.cqG = alloc(64 * 64 * 8);
          h.cqRinv = alloc(64 * 64 * 8);
          h.cqRacc = alloc(64 * 64 * 8);
          h.cqFlag = alloc(4);
          h.cqPart = alloc((size_t)ceil_div(fib, 64) * 64 * 4);
          // pass 1's column digits of H_(n)^T (in cqCol) serve the mode product H x_n P_n^T afterwards,
          // so the later passes slice into buffers of their own
          h.cqCol2 = alloc((size_t)kOzSlices * 64 * ldP * 2);
          h.cqColE2 = alloc(64 * 4);
          h.ozB2 = alloc((size_t)kOzSlices * cols * ldk * 2);
          h.ozEB2 = alloc((size_t)cols * 4);
        }
      }
    }
    if (f32la) {
      int64_t stack_rows = 0;
      for (int m = 0; m < d; ++m) {
        const int64_t rows = Hsz / h.b[m];
        stack_rows = std::max<int64_t>(stack_rows, (int64_t)ceil_div(rows, tsqr_block_rows(plan->bmax)) * h.b[m]);
      }
      h.stk[0] = alloc((size_t)stack_rows * bm * 4);
      h.stk[1] = alloc((size_t)stack_rows * bm * 4);
      h.Wh = alloc(Hsz * 4);
      h.tauh = alloc((size_t)bm * 4);
      h.R32 = alloc((size_t)bm * bm * 4);
      for (int m = 0; m < d; ++m) {
        h.P32[m] = alloc((size_t)h.b[m] * h.rmax[m] * 4);
        h.sv[m] = alloc((size_t)h.b[m] * 4);
      }
    }
  }
  plan->ws_bytes = align_up(ws);

  // ---- launch tables
  plan->lane_p0 = 0;
  plan->lane_p1 = num_problems;
  if (mixed) {
    build_mixed_stages(plan, kron, f32la);
    if (plan->backward_ok) build_backward3_mixed(plan);
  } else {
  std::vector<OmegaJob> om_ext, om_int;
  int64_t om_blocks = 0;
  GemmList gM, gY, gA, gH;
  std::vector<CoreSketchJob> cs;
  int64_t cs_total = 0;
  std::vector<QrJob> qr;
  double cs_flops = 0.0, cs_bytes = 0.0, qr_flops = 0.0, qr_bytes = 0.0;
  std::vector<GemmList> chain(std::max(1, plan->dmax - 1));
  for (int p = 0; p < plan->nprob; ++p) {
    auto& h = plan->probs[p];
    const int d = h.d;
    for (int m = 0; m < d; ++m) {
      OmegaJob oj;
      std::memset(&oj, 0, sizeof(oj));
      oj.out = op(B_OMEGA, h.omega_off[m] * 8);
      oj.count = h.n[m] * h.s[m];
      oj.begin = om_blocks;
      oj.problem = p;
      oj.mode = m;
      oj.bf16 = prm.omega_lowprec != 0;
      om_blocks += (oj.count + 3) / 4;
      om_ext.push_back(oj);
      // (a) M_m = Ucat_m^T Omega_m  (R_m x s_m)
      gM.add(gemm(h.R[m], h.s[m], (int)h.n[m], op_abs(h.factors[m]), h.n[m], 1,
                  op(B_OMEGA, h.omega_off[m] * 8), h.n[m], 1, op(B_WS, h.M[m]), 1, h.R[m]));
    }
    for (int k = 0; k < h.K; ++k) {
      for (int n = 0; n < d; ++n) {
        CoreSketchJob j;
        std::memset(&j, 0, sizeof(j));
        j.core = op_abs(h.cores, (size_t)h.core_off[k] * 8);
        for (int m = 0; m < d; ++m) {
          j.M[m] = op(B_WS, h.M[m]);
          j.r[m] = h.ranks[(size_t)k * d + m];
          j.roff[m] = h.roff[(size_t)k * d + m];
          j.R[m] = h.R[m];
          j.s[m] = h.s[m];
        }
        j.V = op(B_WS, h.V[n]);
        j.d = d;
        j.n = n;
        j.kron = kron;
        j.S = h.S[n];
        j.Rn = h.R[n];
        j.alpha = h.alpha[k];
        j.count = (int64_t)j.r[n] * j.S;
        {
          double other = 1.0;
          for (int m = 0; m < d; ++m)
            if (m != n) other *= j.r[m];
          cs_flops += 2.0 * (double)j.count * other;
          cs_bytes += 8.0 * ((double)j.count * (1.0 + 0.0) + other * j.r[n]);
        }
        j.begin = cs_total;
        cs_total += j.count;
        cs.push_back(j);
      }
    }
    for (int n = 0; n < d; ++n) {
      // (b) Y_n = Ucat_n Vcat_n  (n x S)
      gY.add(gemm((int)h.n[n], h.S[n], h.R[n], op_abs(h.factors[n]), 1, h.n[n], op(B_WS, h.V[n]), h.R[n],
                  1, op(B_Y, h.y_off[n] * 8), 1, h.n[n]));
      QrJob q;
      std::memset(&q, 0, sizeof(q));
      q.Y = op(B_Y, h.y_off[n] * 8);
      q.W = op(B_WS, h.W[n]);
      q.Q = op(B_Q, h.q_off[n] * 8);
      q.tau = op(B_WS, h.tau[n]);
      q.gate = Operand{B_NONE, 0, 0};
      q.n = (int)h.n[n];
      q.S = h.S[n];
      q.b = h.b[n];
      qr.push_back(q);
      qr_flops += 4.0 * (double)h.n[n] * h.b[n] * h.b[n];
      qr_bytes += 8.0 * (double)h.n[n] * (h.S[n] + h.b[n]);
      // (c1) A_n = Q_n^T Ucat_n  (b x R)
      gA.add(gemm(h.b[n], h.R[n], (int)h.n[n], op(B_Q, h.q_off[n] * 8), h.n[n], 1, op_abs(h.factors[n]),
                  h.n[n], 1, op(B_WS, h.A[n]), 1, h.b[n]));
    }
    // (c2) per-term chain T_k = G_k x_1 A_k1 ... x_{d-1} A_k,d-1, last step into Tcat (R_d x P)
    const int Rd = h.R[d - 1];
    for (int k = 0; k < h.K; ++k) {
      const int* r = &h.ranks[(size_t)k * d];
      const int rd_off = h.roff[(size_t)k * d + d - 1];
      for (int t = 0; t + 1 < d; ++t) {
        int64_t L = 1, Rr = 1;
        for (int j = 0; j < t; ++j) L *= h.b[j];
        for (int j = t + 1; j < d; ++j) Rr *= r[j];
        const int I = r[t], Jn = h.b[t];
        const Operand X = (t == 0) ? op_abs(h.cores, (size_t)h.core_off[k] * 8)
                                   : op(B_WS, h.chain[2 * k + ((t - 1) & 1)]);
        const Operand Ablk = op(B_WS, h.A[t] + (size_t)h.b[t] * h.roff[(size_t)k * d + t] * 8);
        const bool last = (t == d - 2);
        const Operand Y = last ? op(B_WS, h.T + (size_t)rd_off * 8) : op(B_WS, h.chain[2 * k + (t & 1)]);
        const double alpha = (t == 0) ? h.alpha[k] : 1.0;
        GemmJob j;
        if (L == 1) {
          // C[j, rr] = sum_i A[j, i] X[i + I rr]
          j = gemm(Jn, (int)Rr, I, Ablk, 1, h.b[t], X, I, 1, Y, last ? Rd : 1, last ? 1 : Jn, alpha);
        } else {
          // C[l, j] = sum_i X[l + L i + L I rr] A[j + b_t i], batched over rr
          j = gemm((int)L, Jn, I, X, 1, L, Ablk, 1, h.b[t], Y, last ? Rd : 1, last ? (int64_t)Rd * L : L, alpha);
          j.batch = (int)Rr;
          j.a_b = L * I;
          j.c_b = last ? 1 : L * Jn;
        }
        chain[t].add(j);
      }
    }
    // (c3) H_(d)^T = Tcat^T A_d^T  (P x b_d), written as the tensor H (mode 1 fastest)
    int64_t Pd = 1;
    for (int j = 0; j + 1 < d; ++j) Pd *= h.b[j];
    gH.add(gemm((int)Pd, h.b[d - 1], Rd, op(B_WS, h.T), Rd, 1, op(B_WS, h.A[d - 1]), 1, h.b[d - 1],
                op(B_H, h.h_off * 8), 1, Pd));
  }
  plan->push(plan->st_omega, S_OMEGA, om_ext, om_blocks, "a1:omega", 0.0, 8.0 * plan->omega_elems);
  // sketch: Omega (workspace) -> M -> V -> Y
  plan->push(plan->st_sketch, S_OMEGA, om_ext, om_blocks, "a1:omega", 0.0, 8.0 * plan->omega_elems);
  plan->push_gemm(plan->st_sketch, gM, "a2:M=UcatT.Omega");
  plan->push(plan->st_sketch, S_CORESKETCH, cs, cs_total, "a3:core_sketch", cs_flops, cs_bytes);
  plan->push_gemm(plan->st_sketch, gY, "a4:Y=Ucat.Vcat");
  // project: A -> chain -> H
  plan->push_gemm(plan->st_project, gA, "a6:A=QT.Ucat");
  for (size_t t = 0; t < chain.size(); ++t) {
    char nm[32];
    std::snprintf(nm, sizeof(nm), "a7:chain%d", (int)t);
    plan->push_gemm(plan->st_project, chain[t], nm);
  }
  plan->push_gemm(plan->st_project, gH, "a8:H=Acat.Tcat");
  // recompress: sketch, QR, project, ST-HOSVD
  plan->st_recompress = plan->st_sketch;
  plan->push(plan->st_recompress, S_QR, qr, (int64_t)qr.size(), "a5:qr", qr_flops, qr_bytes);
  for (const auto& s : plan->st_project) plan->st_recompress.push_back(s);
  if (plan->backward_ok) {
    plan->push_gemm(plan->st_backward, gA, "bwd:A=QT.Ucat");
    build_backward3(plan);
  }
  }
  plan->trunc_from = plan->st_recompress.size();
  {
    std::vector<TruncErrJob> te;
    for (size_t p = 0; p < plan->probs.size(); ++p) {
      TruncErrJob j;
      std::memset(&j, 0, sizeof(j));
      j.err = op(B_WS, plan->probs[p].errw);
      j.out = op(B_OUT, p * sizeof(double));
      j.d = plan->probs[p].d;
      te.push_back(j);
    }
    plan->push(plan->st_truncerr, S_TRUNCERR, te, (int64_t)te.size(), "truncation_error");
  }
  if (f32la) build_hosvd_f32(plan);
  else build_hosvd_f64(plan);

  if (!plan->build_error.empty()) {
    const std::string msg = plan->build_error;
    tks_plan_destroy(plan);
    return fail(TKS_EUNSUPPORTED, msg);
  }

  if (mixed) {
    const int lanes = std::min<int>(prm.lanes, num_problems);
    if (lanes > 1) {
      // one more set of launch tables per group of problems; the full-range lists stay for the
      // other entry points and for profiled calls
      auto om = plan->st_omega, sk = plan->st_sketch, pr = plan->st_project, rc = plan->st_recompress;
      for (int l = 0; l < lanes; ++l) {
        plan->st_omega.clear();
        plan->st_sketch.clear();
        plan->st_project.clear();
        plan->st_recompress.clear();
        plan->lane_p0 = (int)((int64_t)l * num_problems / lanes);
        plan->lane_p1 = (int)((int64_t)(l + 1) * num_problems / lanes);
        build_mixed_stages(plan, kron, f32la);
        if (f32la) build_hosvd_f32(plan);
        else build_hosvd_f64(plan);
        plan->lane_steps.push_back(std::move(plan->st_recompress));
      }
      if (!plan->build_error.empty()) {
        const std::string msg = plan->build_error;
        tks_plan_destroy(plan);
        return fail(TKS_EUNSUPPORTED, msg);
      }
      // a lane's tensor-core GEMMs share the SMs with the other lanes' kernels, some of which hold
      // all 512 TMEM columns of their SM (the persistent digit products, the Gram kernel): one CTA
      // per SM keeps a GEMM CTA from landing beside one of them and waiting for columns
      for (auto& l : plan->lane_steps)
        for (auto& st : l) st.beside_lanes = true;
      plan->st_omega = std::move(om);
      plan->st_sketch = std::move(sk);
      plan->st_project = std::move(pr);
      plan->st_recompress = std::move(rc);
      plan->lane_p0 = 0;
      plan->lane_p1 = num_problems;
      bool ok = cudaEventCreateWithFlags(&plan->lane_fork, cudaEventDisableTiming) == cudaSuccess;
      for (int l = 1; l < lanes && ok; ++l) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        if (ok) plan->lane_streams.push_back(st);
        ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (ok) plan->lane_join.push_back(ev);
      }
      if (!ok) {
        tks_plan_destroy(plan);
        return fail(TKS_ECUDA, "lane streams and events");
      }
    }
  }

  // every launch counts its tiles, blocks or elements in 32 bits
  {
    std::vector<const std::vector<Step>*> lists = {&plan->st_omega,    &plan->st_sketch,   &plan->st_project,
                                                   &plan->st_recompress, &plan->st_backward, &plan->st_truncerr};
    for (const auto& l : plan->lane_steps) lists.push_back(&l);
    for (const auto* l : lists)
      for (const Step& st : *l)
        if (st.work > INT32_MAX) {
          const std::string msg = std::string(st.name) +
                                  ": more than 2^31 - 1 tiles or elements in one launch (split the batch over plans)";
          tks_plan_destroy(plan);
          return fail(TKS_EUNSUPPORTED, msg);
        }
  }

  // ---- device copies
  if (cudaGetDevice(&plan->device) != cudaSuccess) {
    tks_plan_destroy(plan);
    return fail(TKS_ECUDA, "no CUDA device");
  }
  if (plan->bmax > 0 && !f32la) {
    cudaError_t e = prepare_la64(plan->bmax);
    if (e != cudaSuccess) {
      tks_plan_destroy(plan);
      return fail(TKS_ECUDA, std::string("float64 TSQR/SVD shared memory: ") + cudaGetErrorString(e));
    }
  }
  if (f32la) {
    cudaError_t e = prepare_svd_f32(plan->bmax);
    if (e == cudaSuccess) e = prepare_tsqr_f32();
    if (e != cudaSuccess) {
      tks_plan_destroy(plan);
      return fail(TKS_ECUDA, std::string("float32 QR/SVD shared memory: ") + cudaGetErrorString(e));
    }
  }
  if (mixed) {
    cudaError_t e = prepare_tc_gemm();
    if (e == cudaSuccess) e = prepare_order3_kernels();
    if (e == cudaSuccess) e = prepare_proj3();
    if (e == cudaSuccess) e = prepare_fold4();
    if (e == cudaSuccess) e = prepare_sketch3();
    if (e == cudaSuccess) e = prepare_sketch4();
    if (e == cudaSuccess) e = prepare_qr_reg_f32();
    if (e == cudaSuccess) e = prepare_ttm_rows();
    if (e == cudaSuccess) e = prepare_oz_gemm();
    if (e != cudaSuccess) {
      tks_plan_destroy(plan);
      return fail(TKS_ECUDA, std::string("tensor-core GEMM shared memory: ") + cudaGetErrorString(e));
    }
    if (!plan->map_specs.empty()) {
      const size_t bytes = plan->map_specs.size() * sizeof(CUtensorMap);
      plan->maps_off = align_up(plan->arena_host.size(), 128);
      plan->arena_host.resize(plan->maps_off + bytes, 0);
      if (cudaMallocHost(&plan->maps_host, bytes) != cudaSuccess) {
        tks_plan_destroy(plan);
        return fail(TKS_ENOMEM, "pinned tensor-map staging buffer");
      }
    }
  }
  const size_t status_off = plan->add_table(&plan->nprob, 0);
  plan->arena_host.resize(status_off + 64, 0);
  if (cudaMalloc(&plan->arena_dev, plan->arena_host.size()) != cudaSuccess) {
    tks_plan_destroy(plan);
    return fail(TKS_ENOMEM, "descriptor tables");
  }
  if (cudaMemcpy(plan->arena_dev, plan->arena_host.data(), plan->arena_host.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    tks_plan_destroy(plan);
    return fail(TKS_ECUDA, "copying descriptor tables");
  }
  plan->status = reinterpret_cast<Status*>(plan->arena_dev + status_off);
  *out = plan;
  return TKS_OK;
}

tks_status tks_plan_info(const tks_plan* plan, tks_plan_info_t* info) {
  if (!plan || !info) return fail(TKS_EINVAL, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->workspace_bytes = plan->ws_bytes;
  info->omega_elems = plan->omega_elems;
  info->sketch_elems = plan->sketch_elems;
  info->basis_elems = plan->basis_elems;
  info->core_elems = plan->core_elems;
  info->output_elems = plan->output_elems;
  info->num_problems = plan->nprob;
  if (plan->lane_steps.empty()) {
    info->launches_recompress = (int32_t)plan->st_recompress.size();
  } else {
    size_t n = 0;
    for (const auto& ls : plan->lane_steps) n += ls.size();
    info->launches_recompress = (int32_t)n;
  }
  info->flops_lowprec = plan->flops_low;
  info->flops_fp64 = plan->flops_f64;
  info->grad_core_elems = plan->grad_core_elems;
  info->launches_backward = plan->backward_ok ? (int32_t)plan->st_backward.size() : 0;
  info->grad_factor_elems = plan->grad_factor_elems;
  return TKS_OK;
}

tks_status tks_sketch_sizes(int32_t sketch, int32_t order, const int32_t* target_ranks, const int32_t* oversampling,
                            int32_t* omega_cols, int32_t* sketch_cols) {
  if (sketch != TKS_SKETCH_KRON && sketch != TKS_SKETCH_KRP) return fail(TKS_EINVAL, "unknown sketch type");
  if (order < 2 || order > TKS_MAX_ORDER) return fail(TKS_EINVAL, "order out of range");
  if (!target_ranks || !oversampling || !omega_cols || !sketch_cols) return fail(TKS_EINVAL, "null pointer");
  int ell[TKS_MAX_ORDER] = {}, sz[TKS_MAX_ORDER] = {}, cols[TKS_MAX_ORDER] = {};
  for (int m = 0; m < order; ++m) {
    if (target_ranks[m] < 1 || oversampling[m] < 0) return fail(TKS_EINVAL, "bad target/oversampling");
    if ((int64_t)target_ranks[m] + oversampling[m] > kMaxEll) return fail(TKS_EINVAL, "target + oversampling above 2^21");
    ell[m] = target_ranks[m] + oversampling[m];
  }
  const tks_status st = sketch_sizes(sketch, order, ell, sz, cols, "");
  if (st != TKS_OK) return st;
  for (int m = 0; m < order; ++m) {
    omega_cols[m] = sz[m];
    sketch_cols[m] = cols[m];
  }
  return TKS_OK;
}

tks_status tks_problem_info(const tks_plan* plan, int32_t p, tks_problem_info_t* info) {
  if (!plan || !info || p < 0 || p >= plan->nprob) return fail(TKS_EINVAL, "bad plan, problem or info");
  std::memset(info, 0, sizeof(*info));
  const auto& h = plan->probs[p];
  info->order = h.d;
  for (int m = 0; m < h.d; ++m) {
    info->R[m] = h.R[m];
    info->omega_cols[m] = h.s[m];
    info->sketch_cols[m] = h.S[m];
    info->basis_cols[m] = h.b[m];
    info->max_ranks[m] = h.rmax[m];
    info->omega_off[m] = h.omega_off[m];
    info->sketch_off[m] = h.y_off[m];
    info->basis_off[m] = h.q_off[m];
    info->out_factor_off[m] = h.out_fac_off[m];
  }
  info->core_off = h.h_off;
  info->out_core_off = h.out_core_off;
  info->grad_core_off = h.gcore_off;
  for (int m = 0; m < h.d; ++m) info->grad_factor_off[m] = h.gfac_off[m];
  return TKS_OK;
}

}  // extern "C"

namespace {

tks_status run_steps(tks_plan* plan, const std::vector<Step>& steps, const Bases& bases, cudaStream_t stream,
                     bool profile = false) {
  // the tensor-core kernels read TMA tensor maps encoded for one workspace address: refuse to launch
  // them against maps of another workspace (or none), which would hand the TMA unit a stale descriptor
  for (const Step& s : steps)
    if ((s.kind == S_TC || s.kind == S_OZGEMM || s.kind == S_OZGRAM) && plan->maps_ws != bases.p[B_WS])
      return fail(TKS_EINVAL, "internal: tensor maps not encoded for this workspace");
  cudaEvent_t* ev = nullptr;
  if (profile && plan->prof_calls < plan->prof_max_calls) {
    ev = plan->prof_events.data() + (size_t)plan->prof_calls * (steps.size() + 1);
    ++plan->prof_calls;
  }
  for (size_t i = 0; i < steps.size(); ++i) {
    const Step& s = steps[i];
    if (ev) cudaEventRecord(ev[i], stream);
    const void* table = plan->arena_dev + s.table_off;
    switch (s.kind) {
      case S_OMEGA:
        launch_omega(static_cast<const OmegaJob*>(table), s.njobs, s.work, bases, plan->params.seed, stream);
        break;
      case S_GEMM:
        launch_gemm_f64(static_cast<const GemmJob*>(table), s.njobs, (int)s.work, bases, stream);
        break;
      case S_REDUCE:
        launch_splitk_reduce_f64(static_cast<const GemmJob*>(table), s.njobs, s.work, bases, stream);
        break;
      case S_CORESKETCH:
        launch_core_sketch_f64(static_cast<const CoreSketchJob*>(table), s.njobs, s.work, bases, stream);
        break;
      case S_QR:
        launch_qr_f64(static_cast<const QrJob*>(table), s.njobs, bases, plan->status, stream);
        break;
      case S_TSQR64:
        launch_tsqr_f64(static_cast<const TsqrJob*>(table), s.njobs, plan->bmax, bases, stream);
        break;
      case S_SVD64:
        launch_svd_f64(static_cast<const SvdJob*>(table), s.njobs, plan->bmax, bases, plan->status, stream);
        break;
      case S_OZSLICE:
        launch_oz_slice(static_cast<const OzSliceJob*>(table), s.njobs, (int)s.work, bases, stream);
        break;
      case S_OZGEMM:
        launch_oz_gemm(static_cast<const OzGemmJob*>(table), s.njobs, (int)s.work, plan->arena_dev + plan->maps_off,
                       bases, plan->status, plan->wait_cycles, stream);
        break;
      case S_OZXMAX:
        launch_oz_xmax(static_cast<const OzXSliceJob*>(table), s.njobs, (int)s.work, bases, stream);
        break;
      case S_OZXDIG:
        launch_oz_xdig(static_cast<const OzXSliceJob*>(table), s.njobs, (int)s.work, bases, stream);
        break;
      case S_OZGRAM:
        launch_oz_gram(static_cast<const OzGramJob*>(table), s.njobs, plan->arena_dev + plan->maps_off, bases,
                       plan->status, plan->wait_cycles, stream);
        break;
      case S_CHOL:
        launch_chol_step(static_cast<const CholJob*>(table), s.njobs, bases, plan->status, stream);
        break;
      case S_TRUNCERR:
        launch_trunc_err(static_cast<const TruncErrJob*>(table), s.njobs, bases, stream);
        break;
      case S_TTM64:
        launch_ttm_f64(static_cast<const TtmJob*>(table), s.njobs, (int)s.work, s.nb_max, plan->bmax, bases, stream);
        break;
      case S_TC:
        launch_tc_gemm(static_cast<const TcJob*>(table), s.njobs, (int)s.work, plan->arena_dev + plan->maps_off,
                       s.na_max, s.nb_max, bases, plan->status, plan->wait_cycles,
                       plan->stall ? plan->stall_word() : nullptr, plan->params.tc_stages, s.kmax,
                       !s.beside_lanes, stream);
        break;
      case S_SIMT:
        launch_simt_gemm_f32(static_cast<const SimtJob*>(table), s.njobs, (int)s.work, bases, stream);
        break;
      case S_CS32:
        launch_core_sketch_f32(static_cast<const CoreSketchF32Job*>(table), s.njobs, s.work, bases, stream);
        break;
      case S_SPLIT:
        launch_split_f64(static_cast<const SplitJob*>(table), s.njobs, s.work, bases, stream);
        break;
      case S_TRANSPOSE:
        launch_transpose_bf16(static_cast<const TransposeJob*>(table), s.njobs, (int)s.work, bases, stream);
        break;
      case S_QR32:
        launch_qr_f32(static_cast<const QrF32Job*>(table), s.njobs, bases, plan->status, stream);
        break;
      case S_SVD32:
        launch_svd_f32(static_cast<const SvdJob*>(table), s.njobs, plan->bmax, bases, plan->status, stream);
        break;
      case S_TSQR:
        launch_tsqr_f32(static_cast<const TsqrJob*>(table), s.njobs, tsqr_block_rows(plan->bmax), plan->bmax, bases,
                        stream);
        break;
      case S_TTM:
        launch_ttm_rows(static_cast<const TtmJob*>(table), s.njobs, (int)s.work, bases, stream);
        break;
      case S_QRREG:
        launch_qr_reg_f32(static_cast<const QrF32Job*>(table), s.njobs, (int)s.work, s.smem, bases, plan->status,
                          stream);
        break;
      case S_QRSM:
        launch_qr_smem_f32(static_cast<const QrF32Job*>(table), s.njobs, s.smem, bases, plan->status, stream);
        break;
      case S_CS3:
        launch_core_sketch_krp3(static_cast<const CoreSketchF32Job*>(table), s.njobs, s.smem, bases, stream);
        break;
      case S_CHAIN3:
        launch_chain3(static_cast<const Chain3Job*>(table), s.njobs, s.smem, bases, stream);
        break;
      case S_SK3:
        launch_sketch3(static_cast<const Sketch3Job*>(table), s.njobs, s.smem, bases, plan->status, stream);
        break;
      case S_SK4:
        launch_sketch4(static_cast<const Sketch4Job*>(table), s.njobs, s.smem, bases, stream);
        break;
      case S_SK3F:
        launch_sketch3(static_cast<const Sketch3Job*>(table), s.njobs, s.smem, bases, plan->status, stream);
        break;
      case S_PROJ3:
        launch_proj3(static_cast<const Proj3Job*>(table), s.njobs, false, bases, plan->status, stream);
        break;
      case S_PROJ3F:
        launch_proj3(static_cast<const Proj3Job*>(table), s.njobs, true, bases, plan->status, stream);
        break;
      case S_FOLD4:
        launch_fold4(static_cast<const Fold4Job*>(table), s.njobs, s.smem, bases, stream);
        break;
    }
  }
  if (ev) cudaEventRecord(ev[steps.size()], stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(TKS_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return TKS_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Encodes the plan's TMA tensor maps for this workspace pointer (bf16, 2-D, 64-element
// (128-byte) inner box with 128-byte swizzle, zero fill out of bounds) and copies them to the
// device table on `stream`; reused while the same workspace is passed.
tks_status ensure_maps(tks_plan* plan, void* ws, cudaStream_t stream) {
  if (plan->map_specs.empty() || plan->maps_ws == ws) return TKS_OK;
  auto enc = tensor_map_encoder();
  if (!enc) return fail(TKS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (plan->maps_pending) TKS_CUDA_CHECK(cudaStreamSynchronize(stream));
  auto* maps = static_cast<CUtensorMap*>(plan->maps_host);
  for (size_t i = 0; i < plan->map_specs.size(); ++i) {
    const auto& m = plan->map_specs[i];
    void* base = (m.base == B_ABS) ? reinterpret_cast<void*>(m.off) : static_cast<char*>(ws) + m.off;
    cuuint64_t dims[2] = {m.K, m.rows};
    cuuint64_t strides[1] = {m.ld * 2};
    cuuint32_t box[2] = {64, m.box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&maps[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TKS_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  }
  TKS_CUDA_CHECK(cudaMemcpyAsync(plan->arena_dev + plan->maps_off, plan->maps_host,
                                 plan->map_specs.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, stream));
  plan->maps_ws = ws;
  plan->maps_pending = true;
  return TKS_OK;
}

Bases bind(tks_plan* plan, void* ws) {
  Bases b;
  std::memset(&b, 0, sizeof(b));
  char* w = static_cast<char*>(ws);
  b.p[B_WS] = w;
  b.p[B_OMEGA] = w + plan->ws_omega;
  b.p[B_Y] = w + plan->ws_Y;
  b.p[B_Q] = w + plan->ws_Q;
  b.p[B_H] = w + plan->ws_H;
  return b;
}

tks_status check_ws(tks_plan* plan, void* ws) {
  if (!plan) return fail(TKS_EINVAL, "null plan");
  if (!ws && plan->ws_bytes > 0) return fail(TKS_EINVAL, "null workspace");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(TKS_EINVAL, "workspace not 256-byte aligned");
  return TKS_OK;
}

}  // namespace

extern "C" {

tks_status tks_generate_omega(tks_plan* plan, void* workspace, double* omega_out, void* stream) {
  tks_status st = check_ws(plan, workspace);
  if (st != TKS_OK) return st;
  if (!omega_out) return fail(TKS_EINVAL, "null omega_out");
  Bases b = bind(plan, workspace);
  b.p[B_OMEGA] = reinterpret_cast<char*>(omega_out);
  return run_steps(plan, plan->st_omega, b, static_cast<cudaStream_t>(stream));
}

tks_status tucker_sum_sketch(tks_plan* plan, void* workspace, double* Y_out, void* stream) {
  tks_status st = check_ws(plan, workspace);
  if (st != TKS_OK) return st;
  if (!Y_out) return fail(TKS_EINVAL, "null Y_out");
  st = ensure_maps(plan, workspace, static_cast<cudaStream_t>(stream));
  if (st != TKS_OK) return st;
  Bases b = bind(plan, workspace);
  b.p[B_Y] = reinterpret_cast<char*>(Y_out);
  return run_steps(plan, plan->st_sketch, b, static_cast<cudaStream_t>(stream));
}

tks_status tks_project_core(tks_plan* plan, void* workspace, const double* Q_in, double* H_out, void* stream) {
  tks_status st = check_ws(plan, workspace);
  if (st != TKS_OK) return st;
  if (!Q_in || !H_out) return fail(TKS_EINVAL, "null Q_in or H_out");
  st = ensure_maps(plan, workspace, static_cast<cudaStream_t>(stream));
  if (st != TKS_OK) return st;
  Bases b = bind(plan, workspace);
  b.p[B_Q] = reinterpret_cast<char*>(const_cast<double*>(Q_in));
  b.p[B_H] = reinterpret_cast<char*>(H_out);
  return run_steps(plan, plan->st_project, b, static_cast<cudaStream_t>(stream));
}

tks_status tucker_sum_recompress(tks_plan* plan, void* workspace, double* out, int32_t* ranks_out, void* stream) {
  tks_status st = check_ws(plan, workspace);
  if (st != TKS_OK) return st;
  if (!out || !ranks_out) return fail(TKS_EINVAL, "null out or ranks_out");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = ensure_maps(plan, workspace, s);
  if (st != TKS_OK) return st;
  TKS_CUDA_CHECK(cudaMemsetAsync(ranks_out, 0, (size_t)plan->nprob * TKS_MAX_ORDER * sizeof(int32_t), s));
  TKS_CUDA_CHECK(cudaMemsetAsync(out, 0, (size_t)plan->output_elems * sizeof(double), s));
  Bases b = bind(plan, workspace);
  b.p[B_OUT] = reinterpret_cast<char*>(out);
  b.p[B_RANKS] = reinterpret_cast<char*>(ranks_out);
  const bool profiled = plan->prof_calls < plan->prof_max_calls;
  if (plan->lane_steps.empty() || profiled) return run_steps(plan, plan->st_recompress, b, s, true);
  // fork: every extra lane waits for the caller's stream, runs its problems, and is joined back
  TKS_CUDA_CHECK(cudaEventRecord(plan->lane_fork, s));
  for (cudaStream_t ls : plan->lane_streams) TKS_CUDA_CHECK(cudaStreamWaitEvent(ls, plan->lane_fork, 0));
  for (size_t l = 0; l < plan->lane_steps.size(); ++l) {
    st = run_steps(plan, plan->lane_steps[l], b, l == 0 ? s : plan->lane_streams[l - 1], false);
    if (st != TKS_OK) return st;
  }
  for (size_t l = 1; l < plan->lane_steps.size(); ++l) {
    TKS_CUDA_CHECK(cudaEventRecord(plan->lane_join[l - 1], plan->lane_streams[l - 1]));
    TKS_CUDA_CHECK(cudaStreamWaitEvent(s, plan->lane_join[l - 1], 0));
  }
  return TKS_OK;
}

tks_status tks_truncate_core(tks_plan* plan, void* workspace, const double* Q_in, const double* H_in, double* out,
                             int32_t* ranks_out, void* stream) {
  tks_status st = check_ws(plan, workspace);
  if (st != TKS_OK) return st;
  if (!Q_in || !H_in || !out || !ranks_out) return fail(TKS_EINVAL, "null Q_in, H_in, out or ranks_out");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = ensure_maps(plan, workspace, s);
  if (st != TKS_OK) return st;
  TKS_CUDA_CHECK(cudaMemsetAsync(ranks_out, 0, (size_t)plan->nprob * TKS_MAX_ORDER * sizeof(int32_t), s));
  TKS_CUDA_CHECK(cudaMemsetAsync(out, 0, (size_t)plan->output_elems * sizeof(double), s));
  Bases b = bind(plan, workspace);
  b.p[B_Q] = reinterpret_cast<char*>(const_cast<double*>(Q_in));
  b.p[B_H] = reinterpret_cast<char*>(const_cast<double*>(H_in));
  b.p[B_OUT] = reinterpret_cast<char*>(out);
  b.p[B_RANKS] = reinterpret_cast<char*>(ranks_out);
  const std::vector<Step> steps(plan->st_recompress.begin() + (std::ptrdiff_t)plan->trunc_from,
                                plan->st_recompress.end());
  return run_steps(plan, steps, b, s);
}

tks_status tks_profile_begin(tks_plan* plan, int32_t max_calls) {
  if (!plan || max_calls < 1) return fail(TKS_EINVAL, "bad plan or max_calls");
  plan->profile_clear();
  const size_t n = (size_t)max_calls * (plan->st_recompress.size() + 1);
  plan->prof_events.resize(n);
  for (size_t i = 0; i < n; ++i) {
    if (cudaEventCreate(&plan->prof_events[i]) != cudaSuccess) {
      plan->prof_events.resize(i);
      plan->profile_clear();
      return fail(TKS_ECUDA, "cudaEventCreate");
    }
  }
  plan->prof_max_calls = max_calls;
  plan->prof_calls = 0;
  return TKS_OK;
}

tks_status tks_profile_end(tks_plan* plan, tks_step_profile_t* out, int32_t cap, int32_t* nsteps) {
  if (!plan || !nsteps) return fail(TKS_EINVAL, "bad plan or nsteps");
  const size_t ns = plan->st_recompress.size();
  *nsteps = (int32_t)ns;
  const int calls = plan->prof_calls;
  if (calls > 0) {
    cudaError_t e = cudaEventSynchronize(plan->prof_events[(size_t)calls * (ns + 1) - 1]);
    if (e != cudaSuccess) {
      plan->profile_clear();
      return fail(TKS_ECUDA, std::string("cudaEventSynchronize: ") + cudaGetErrorString(e));
    }
  }
  for (size_t i = 0; i < ns && out && (int32_t)i < cap; ++i) {
    const Step& s = plan->st_recompress[i];
    tks_step_profile_t& o = out[i];
    std::memset(&o, 0, sizeof(o));
    std::snprintf(o.name, sizeof(o.name), "%s", s.name);
    o.kind = (int32_t)s.kind;
    o.calls = calls;
    o.flops = s.flops;
    o.bytes = s.bytes;
    double ms = 0.0;
    for (int c = 0; c < calls; ++c) {
      float t = 0.f;
      cudaEventElapsedTime(&t, plan->prof_events[(size_t)c * (ns + 1) + i],
                           plan->prof_events[(size_t)c * (ns + 1) + i + 1]);
      ms += t;
    }
    o.ms = ms;
  }
  plan->profile_clear();
  return TKS_OK;
}

namespace {

std::string knobs_json(const tks_params& p) {
  char b[160];
  std::snprintf(b, sizeof(b), "{\"lanes\": %d, \"sketch_qr\": %d, \"hosvd_r\": %d, \"proj_chunk\": %d, \"tc_stages\": %d}",
                p.lanes, p.sketch_qr, p.hosvd_r, p.proj_chunk, p.tc_stages);
  return b;
}

// Median of three timed recompressions after one untimed call (ms), or a negative value when the
// schedule failed (an error status, a device fault report or a CUDA error).
double time_schedule(tks_plan* plan, void* ws, double* out, int32_t* ranks, cudaStream_t st) {
  if (tucker_sum_recompress(plan, ws, out, ranks, st) != TKS_OK) return -1.0;
  if (tks_sync_status(plan, st) != TKS_OK) return -1.0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return -1.0;
  }
  float t[3] = {0.f, 0.f, 0.f};
  bool ok = true;
  for (int i = 0; i < 3 && ok; ++i) {
    ok = cudaEventRecord(a, st) == cudaSuccess && tucker_sum_recompress(plan, ws, out, ranks, st) == TKS_OK &&
         cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
         cudaEventElapsedTime(&t[i], a, b) == cudaSuccess;
  }
  ok = ok && tks_sync_status(plan, st) == TKS_OK;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (!ok) return -1.0;
  std::sort(t, t + 3);
  return t[1];
}

// Greedy search from the rule: lanes first, then each schedule knob in turn, a second round when the
// first changed anything; a candidate replaces the current pick only when it is at least 2% faster.
// Scratch buffers grow with the largest workspace.
tks_status autotune_plan(tks_plan** out, const tks_problem* problems, int32_t num_problems, const tks_params& prm) {
  tks_params cur = prm;
  cur.autotune = 0;
  tks_plan* best = nullptr;
  tks_status st = create_plan(&best, problems, num_problems, &cur);
  if (st != TKS_OK) return st;
  if (prm.precision == TKS_FP64) {
    best->tuning_rule = cur;
    *out = best;
    return TKS_OK;
  }
  void* ws = nullptr;
  double* o = nullptr;
  int32_t* rk = nullptr;
  size_t ws_cap = 0;
  cudaStream_t stream = nullptr;
  auto cleanup = [&]() {
    if (ws) cudaFree(ws);
    if (o) cudaFree(o);
    if (rk) cudaFree(rk);
    if (stream) cudaStreamDestroy(stream);
  };
  auto ensure_ws = [&](size_t bytes) {
    if (bytes <= ws_cap) return true;
    if (ws) cudaFree(ws);
    ws = nullptr;
    ws_cap = 0;
    if (cudaMalloc(&ws, bytes) != cudaSuccess) return false;
    ws_cap = bytes;
    return true;
  };
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&o), (size_t)std::max<int64_t>(1, best->output_elems) * 8) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&rk), (size_t)num_problems * TKS_MAX_ORDER * 4) != cudaSuccess ||
      !ensure_ws(std::max<size_t>(best->ws_bytes, 256))) {
    cleanup();
    tks_plan_destroy(best);
    return fail(TKS_ENOMEM, "autotune scratch buffers");
  }
  double best_ms = time_schedule(best, ws, o, rk, stream);
  if (best_ms < 0.0) {
    cleanup();
    tks_plan_destroy(best);
    return fail(TKS_ECUDA, "autotune: the rule schedule failed");
  }
  const double rule_ms = best_ms;
  const tks_params rule = cur;
  std::string cand = "[{\"knobs\": " + knobs_json(cur) + ", \"ms\": " + std::to_string(best_ms) + "}";
  const bool f32la = prm.precision == TKS_MIXED_F32LA;
  std::vector<std::pair<int32_t tks_params::*, std::vector<int32_t>>> knobs;
  std::vector<int32_t> lane_opts;
  for (int l = 1; l <= 4 && l <= num_problems; ++l) lane_opts.push_back(l);
  knobs.push_back({&tks_params::lanes, lane_opts});
  if (!f32la) {
    knobs.push_back({&tks_params::sketch_qr, {0, 3, 2}});
    knobs.push_back({&tks_params::hosvd_r, {0, 3, 2}});
  }
  knobs.push_back({&tks_params::proj_chunk, {0, 8}});
  knobs.push_back({&tks_params::tc_stages, {0, 3, 2}});
  // coordinate descent: a second round revisits every knob once the first changed any
  for (int round = 0; round < 2; ++round) {
    const tks_params before = cur;
    for (const auto& kv : knobs) {
      const int32_t picked = cur.*(kv.first);
      for (int32_t v : kv.second) {
        if (v == picked || (kv.first == &tks_params::lanes && v <= 1 && picked <= 1)) continue;
        tks_params c = cur;
        c.*(kv.first) = v;
        tks_plan* cp = nullptr;
        if (create_plan(&cp, problems, num_problems, &c) != TKS_OK) continue;
        double ms = -1.0;
        if (ensure_ws(std::max<size_t>(cp->ws_bytes, 256))) ms = time_schedule(cp, ws, o, rk, stream);
        cand += ", {\"knobs\": " + knobs_json(c) + ", \"ms\": " + std::to_string(ms) + "}";
        if (ms > 0.0 && ms < 0.98 * best_ms) {
          tks_plan_destroy(best);
          best = cp;
          best_ms = ms;
          cur = c;
        } else {
          tks_plan_destroy(cp);
        }
      }
    }
    if (std::memcmp(&before, &cur, sizeof(cur)) == 0) break;
  }
  cleanup();
  cand += "]";
  best->autotuned = true;
  best->tuning_candidates = cand;
  best->tuning_rule = rule;
  best->tuning_rule_ms = rule_ms;
  best->tuning_picked_ms = best_ms;
  *out = best;
  return TKS_OK;
}

}  // namespace

extern "C" {

tks_status tks_plan_create(tks_plan** out, const tks_problem* problems, int32_t num_problems,
                           const tks_params* params) {
  if (!out) return fail(TKS_EINVAL, "plan output pointer is NULL");
  *out = nullptr;
  if (!params) return fail(TKS_EINVAL, "no params");
  if (params->autotune == 1) return autotune_plan(out, problems, num_problems, *params);
  tks_status st = create_plan(out, problems, num_problems, params);
  if (st == TKS_OK) (*out)->tuning_rule = *params;
  return st;
}

tks_status tks_plan_tuning(const tks_plan* plan, char* buf, int64_t cap, int64_t* len) {
  if (!plan || !len || (cap > 0 && !buf)) return fail(TKS_EINVAL, "null plan, len or buf");
  std::string j = std::string("{\"autotuned\": ") + (plan->autotuned ? "1" : "0") +
                  ", \"picked\": " + knobs_json(plan->params) + ", \"rule\": " + knobs_json(plan->tuning_rule) +
                  ", \"rule_ms\": " + std::to_string(plan->tuning_rule_ms) +
                  ", \"picked_ms\": " + std::to_string(plan->tuning_picked_ms) +
                  ", \"candidates\": " + (plan->tuning_candidates.empty() ? "[]" : plan->tuning_candidates) + "}";
  *len = (int64_t)j.size();
  if (cap > 0) {
    const size_t n = std::min<size_t>((size_t)cap - 1, j.size());
    std::memcpy(buf, j.data(), n);
    buf[n] = '\0';
  }
  return TKS_OK;
}

}  // extern "C"

tks_status tks_truncation_error(tks_plan* plan, void* workspace, double* err_out, void* stream) {
  tks_status st = check_ws(plan, workspace);
  if (st != TKS_OK) return st;
  if (!err_out) return fail(TKS_EINVAL, "null err_out");
  Bases b = bind(plan, workspace);
  b.p[B_OUT] = reinterpret_cast<char*>(err_out);
  return run_steps(plan, plan->st_truncerr, b, static_cast<cudaStream_t>(stream));
}

tks_status tks_project_core_backward(tks_plan* plan, void* workspace, const double* Q_in, const double* Hbar_in,
                                     double* dcores, double* dfactors, void* stream) {
  tks_status st = check_ws(plan, workspace);
  if (st != TKS_OK) return st;
  if (!plan->backward_ok)
    return fail(TKS_EUNSUPPORTED, "tks_project_core_backward needs a plan of order-3 problems");
  if (!Q_in || !Hbar_in || !dcores || !dfactors) return fail(TKS_EINVAL, "null Q_in, Hbar_in, dcores or dfactors");
  st = ensure_maps(plan, workspace, static_cast<cudaStream_t>(stream));
  if (st != TKS_OK) return st;
  Bases b = bind(plan, workspace);
  b.p[B_Q] = reinterpret_cast<char*>(const_cast<double*>(Q_in));
  b.p[B_HBAR] = reinterpret_cast<char*>(const_cast<double*>(Hbar_in));
  b.p[B_DCORE] = reinterpret_cast<char*>(dcores);
  b.p[B_DFAC] = reinterpret_cast<char*>(dfactors);
  return run_steps(plan, plan->st_backward, b, static_cast<cudaStream_t>(stream));
}

tks_status tks_plan_set_fault_test(tks_plan* plan, int64_t wait_cycles, int32_t stall) {
  if (!plan) return fail(TKS_EINVAL, "null plan");
  if (wait_cycles < 0 || (stall != 0 && stall != 1)) return fail(TKS_EINVAL, "wait_cycles < 0 or stall not 0/1");
  plan->wait_cycles = wait_cycles > 0 ? (long long)wait_cycles : kDefaultWaitCycles;
  plan->stall = stall;
  return TKS_OK;
}

tks_status tks_sync_status(tks_plan* plan, void* stream) {
  if (!plan) return fail(TKS_EINVAL, "null plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TKS_CUDA_CHECK(cudaStreamSynchronize(s));
  Status h{0, 0};
  TKS_CUDA_CHECK(cudaMemcpy(&h, plan->status, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.code != 0) {
    const Status zero{0, 0};
    TKS_CUDA_CHECK(cudaMemcpy(plan->status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    return fail(static_cast<tks_status>(h.code), std::string("device reported ") +
                                                     tks_status_string(static_cast<tks_status>(h.code)));
  }
  return TKS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Allocation-free structured sketch of one problem (FP64).  Its descriptor tables and scratch
// live in this file-scope device array; host code only ever uses the address returned by
// cudaGetSymbolAddress for the current device (the symbol itself is a host-side stand-in).
static __device__ __align__(256) unsigned char g_noalloc_scratch[TKS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mutex;
// per device: the context the address was looked up in, and the address itself (a destroyed
// context, e.g. after cudaDeviceReset, reloads the module at another address)
CUcontext g_noalloc_ctx[kMaxDevices] = {};
void* g_noalloc_ptr[kMaxDevices] = {};

typedef CUresult (*PFN_ctx_get_current)(CUcontext*);

PFN_ctx_get_current ctx_get_current() {
  static PFN_ctx_get_current fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_ctx_get_current>(p);
  }
  return fn;
}

tks_status noalloc_scratch(void** out) {
  int dev = -1;
  TKS_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(TKS_EUNSUPPORTED, "device ordinal out of range");
  TKS_CUDA_CHECK(cudaSetDevice(dev));   // initializes the device's primary context and makes it current
  auto get_ctx = ctx_get_current();
  if (!get_ctx) return fail(TKS_ECUDA, "cuCtxGetCurrent is not available from the driver");
  CUcontext ctx = nullptr;
  if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return fail(TKS_ECUDA, "no current CUDA context");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev] || g_noalloc_ctx[dev] != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(TKS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
    g_noalloc_ctx[dev] = ctx;
  }
  *out = g_noalloc_ptr[dev];
  return TKS_OK;
}

struct HostTables {
  std::vector<char> bytes;
  template <typename T>
  size_t add(const std::vector<T>& v) {
    const size_t off = align_up(bytes.size(), 64);
    bytes.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

}  // namespace

extern "C" tks_status tucker_sum_sketch_noalloc(const tks_problem* problem, const tks_params* params, double* Y_out,
                                                void* stream) {
  if (!problem || !params || !Y_out) return fail(TKS_EINVAL, "null problem, params or Y_out");
  if (params->precision != TKS_FP64 || params->dtype != TKS_DT_F64)
    return fail(TKS_EINVAL, "tucker_sum_sketch_noalloc needs TKS_FP64 with float64 inputs");
  if (params->sketch != TKS_SKETCH_KRP && params->sketch != TKS_SKETCH_KRON) return fail(TKS_EINVAL, "bad sketch");
  if (params->omega_lowprec != 0 && params->omega_lowprec != 1)
    return fail(TKS_EINVAL, "omega_lowprec must be 0 or 1");
  if (params->lanes < 0 || params->lanes > 8) return fail(TKS_EINVAL, "lanes must be 0..8");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    // the tables are copied from host memory that lives only during this call
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(TKS_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    }
    if (cs != cudaStreamCaptureStatusNone)
      return fail(TKS_EUNSUPPORTED, "tucker_sum_sketch_noalloc cannot be enqueued while its stream is being captured");
  }
  ProbHost h;
  tks_status st = validate_and_size(*problem, *params, h, 0);
  if (st != TKS_OK) return st;
  const int d = h.d;
  const int kron = params->sketch == TKS_SKETCH_KRON;
  // scratch layout after the tables: Omega_m, M_m, Vcat_n (float64)
  size_t ws = 0;
  auto alloc = [&](size_t bytes) {
    const size_t o = ws;
    ws = align_up(ws + std::max<size_t>(bytes, 1));
    return o;
  };
  int64_t y_off = 0;
  size_t om[MAXD], Mw[MAXD], Vw[MAXD];
  for (int m = 0; m < d; ++m) {
    om[m] = alloc((size_t)h.n[m] * h.s[m] * 8);
    Mw[m] = alloc((size_t)h.R[m] * h.s[m] * 8);
    Vw[m] = alloc((size_t)h.R[m] * h.S[m] * 8);
    h.y_off[m] = y_off;
    y_off += h.n[m] * h.S[m];
  }
  std::vector<OmegaJob> omj;
  int64_t om_blocks = 0;
  GemmList gM, gY;
  std::vector<CoreSketchJob> cs;
  int64_t cs_total = 0;
  for (int m = 0; m < d; ++m) {
    OmegaJob oj;
    std::memset(&oj, 0, sizeof(oj));
    oj.out = op(B_WS, om[m]);
    oj.count = h.n[m] * h.s[m];
    oj.begin = om_blocks;
    oj.problem = 0;
    oj.mode = m;
    oj.bf16 = params->omega_lowprec != 0;
    om_blocks += (oj.count + 3) / 4;
    omj.push_back(oj);
    gM.add(gemm(h.R[m], h.s[m], (int)h.n[m], op_abs(h.factors[m]), h.n[m], 1, op(B_WS, om[m]), h.n[m], 1,
                op(B_WS, Mw[m]), 1, h.R[m]));
  }
  for (int k = 0; k < h.K; ++k) {
    for (int n = 0; n < d; ++n) {
      CoreSketchJob j;
      std::memset(&j, 0, sizeof(j));
      j.core = op_abs(h.cores, (size_t)h.core_off[k] * 8);
      for (int m = 0; m < d; ++m) {
        j.M[m] = op(B_WS, Mw[m]);
        j.r[m] = h.ranks[(size_t)k * d + m];
        j.roff[m] = h.roff[(size_t)k * d + m];
        j.R[m] = h.R[m];
        j.s[m] = h.s[m];
      }
      j.V = op(B_WS, Vw[n]);
      j.d = d;
      j.n = n;
      j.kron = kron;
      j.S = h.S[n];
      j.Rn = h.R[n];
      j.alpha = h.alpha[k];
      j.count = (int64_t)j.r[n] * j.S;
      j.begin = cs_total;
      cs_total += j.count;
      cs.push_back(j);
    }
  }
  for (int n = 0; n < d; ++n)
    gY.add(gemm((int)h.n[n], h.S[n], h.R[n], op_abs(h.factors[n]), 1, h.n[n], op(B_WS, Vw[n]), h.R[n], 1,
                op(B_Y, h.y_off[n] * 8), 1, h.n[n]));
  HostTables t;
  const size_t t_om = t.add(omj), t_gM = t.add(gM.jobs), t_cs = t.add(cs), t_gY = t.add(gY.jobs);
  const size_t tables = align_up(t.bytes.size());
  const size_t need = tables + ws;
  if (need > TKS_NOALLOC_SCRATCH_BYTES)
    return fail(TKS_EINVAL, "tucker_sum_sketch_noalloc: problem needs " + std::to_string(need) +
                                " bytes of scratch, the static scratch holds " +
                                std::to_string((size_t)TKS_NOALLOC_SCRATCH_BYTES));
  void* scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st != TKS_OK) return st;
  char* base = static_cast<char*>(scratch);
  TKS_CUDA_CHECK(cudaMemcpyAsync(base, t.bytes.data(), t.bytes.size(), cudaMemcpyHostToDevice, s));
  Bases b;
  std::memset(&b, 0, sizeof(b));
  b.p[B_WS] = base + tables;
  b.p[B_Y] = reinterpret_cast<char*>(Y_out);
  launch_omega(reinterpret_cast<const OmegaJob*>(base + t_om), (int)omj.size(), om_blocks, b, params->seed, s);
  launch_gemm_f64(reinterpret_cast<const GemmJob*>(base + t_gM), (int)gM.jobs.size(), (int)gM.tiles, b, s);
  launch_core_sketch_f64(reinterpret_cast<const CoreSketchJob*>(base + t_cs), (int)cs.size(), cs_total, b, s);
  launch_gemm_f64(reinterpret_cast<const GemmJob*>(base + t_gY), (int)gY.jobs.size(), (int)gY.tiles, b, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(TKS_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return TKS_OK;
}

namespace tks {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace tks

// C ABI of the effective subrank heuristic (Alg. 5): validation, workspace layout and launch
// tables at plan time; one execute call enqueues the four launches of subrank.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "tks.h"
#include "tks_internal.h"

using namespace tks;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

tks_status fail(tks_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

#define SR_CUDA_CHECK(call)                                                                   \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(TKS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

Operand op_ws(size_t off) { return Operand{B_WS, 0, (int64_t)off}; }
Operand op_base(int32_t base, size_t off) { return Operand{base, 0, (int64_t)off}; }
Operand op_abs(const void* p, size_t off = 0) {
  return Operand{B_ABS, 0, (int64_t)(reinterpret_cast<uintptr_t>(p) + off)};
}

struct MatHost {
  int p, mode, m, R;
  int64_t n;
  bool aat;
  size_t gram, d, e, ev_ws, wcol;
  int64_t ev_off;   // element offset in the eigenvalue buffer
};

}  // namespace

struct tks_subrank_plan {
  int nprob = 0;
  int max_m = 0;
  double eps = 0.0;
  std::vector<MatHost> mats;               // one per (problem, mode), problem-major
  std::vector<int> order;                  // problem orders
  char* arena = nullptr;                   // device: job tables + status word
  size_t off_w = 0, off_g = 0, off_s = 0;  // job tables in the arena
  int nw = 0, ng = 0, ns = 0, gram_tiles = 0;
  Status* status = nullptr;
  size_t ws_bytes = 0, ws_ev = 0;
  int64_t eval_elems = 0;
  double flops = 0.0, gram_flops = 0.0;
  std::vector<int> job_m;                  // order of each tridiagonalization job's matrix
  int32_t* steps = nullptr;                // device: executed reduction steps per job (in the arena)
};

extern "C" {

tks_status tks_subrank_plan_create(tks_subrank_plan** out, const tks_problem* problems, int32_t num_problems,
                                   const tks_params* params) {
  if (!out) return fail(TKS_EINVAL, "plan output pointer is NULL");
  *out = nullptr;
  if (!problems || !params || num_problems < 1) return fail(TKS_EINVAL, "no problems or params");
  const tks_params prm = *params;
  if (!(prm.trunc_tol > 0.0) || !std::isfinite(prm.trunc_tol))
    return fail(TKS_EINVAL, "the subrank heuristic needs a tolerance trunc_tol > 0");
  if (prm.dtype != TKS_DT_F64 && prm.dtype != TKS_DT_BF16) return fail(TKS_EINVAL, "bad dtype");
  const int32_t type = prm.dtype == TKS_DT_BF16 ? T_BF16 : T_F64;
  const size_t esize = prm.dtype == TKS_DT_BF16 ? 2 : 8;

  auto* plan = new tks_subrank_plan();
  plan->nprob = num_problems;
  plan->eps = prm.trunc_tol;
  std::vector<WeightJob> wjobs;
  std::vector<GramJob> gjobs;
  size_t ws = 0;
  auto alloc = [&](size_t bytes) {
    const size_t o = ws;
    ws = align_up(ws + std::max<size_t>(bytes, 1));
    return o;
  };
  auto reject = [&](tks_status st, const std::string& msg) {
    delete plan;
    return fail(st, msg);
  };
  for (int p = 0; p < num_problems; ++p) {
    const tks_problem& P = problems[p];
    const std::string who = "problem " + std::to_string(p) + ": ";
    const int d = P.order;
    if (d < 2 || d > TKS_MAX_ORDER) return reject(TKS_EINVAL, who + "order must be 2..6");
    if (P.num_terms < 1 || !P.dims || !P.ranks || !P.oversampling || !P.cores || !P.factors)
      return reject(TKS_EINVAL, who + "missing dims, ranks, oversampling, cores or factors");
    const int K = P.num_terms;
    int R[MAXD] = {};
    for (int m = 0; m < d; ++m) {
      if (P.dims[m] < 1) return reject(TKS_EINVAL, who + "dims must be >= 1");
      if (P.oversampling[m] < 0) return reject(TKS_EINVAL, who + "oversampling must be >= 0");
      if (!P.factors[m]) return reject(TKS_EINVAL, who + "factor pointer is NULL");
    }
    for (int k = 0; k < K; ++k)
      for (int m = 0; m < d; ++m) {
        const int r = P.ranks[k * d + m];
        if (r < 1 || r > TKS_MAX_RANK || r > P.dims[m])
          return reject(TKS_EINVAL, who + "term ranks must be in 1..min(n_m, 64)");
        R[m] += r;
      }
    if (P.alpha)
      for (int k = 0; k < K; ++k)
        if (!std::isfinite(P.alpha[k])) return reject(TKS_EINVAL, who + "alpha must be finite");
    size_t wcol[MAXD];
    for (int m = 0; m < d; ++m) wcol[m] = alloc(sizeof(double) * R[m]);
    // term weights
    int64_t core_off = 0;
    int roff[MAXD] = {};
    for (int k = 0; k < K; ++k) {
      WeightJob j;
      std::memset(&j, 0, sizeof(j));
      int64_t cnt = 1;
      for (int m = 0; m < d; ++m) cnt *= P.ranks[k * d + m];
      j.core = op_abs(P.cores, (size_t)core_off * esize);
      j.count = cnt;
      j.type = type;
      j.d = d;
      for (int m = 0; m < d; ++m) {
        j.r[m] = P.ranks[k * d + m];
        j.wcol[m] = op_ws(wcol[m] + sizeof(double) * roff[m]);
        roff[m] += j.r[m];
      }
      j.alpha = P.alpha ? P.alpha[k] : 1.0;
      wjobs.push_back(j);
      core_off += cnt;
    }
    // one Gram matrix per mode
    for (int m = 0; m < d; ++m) {
      MatHost h;
      h.p = p;
      h.mode = m;
      h.n = P.dims[m];
      h.R = R[m];
      h.aat = (int64_t)R[m] > P.dims[m];
      h.m = h.aat ? (int)P.dims[m] : R[m];
      if (h.m > kSubrankMaxDim)
        return reject(TKS_EUNSUPPORTED, who + "min(n_m, R_m) = " + std::to_string(h.m) + " exceeds " +
                                            std::to_string(kSubrankMaxDim));
      h.wcol = wcol[m];
      h.gram = alloc(sizeof(double) * (size_t)h.m * h.m);
      h.d = alloc(sizeof(double) * h.m);
      h.e = alloc(sizeof(double) * h.m);
      h.ev_off = plan->eval_elems;
      plan->eval_elems += h.m;
      plan->max_m = std::max(plan->max_m, h.m);
      const int T = (h.m + 63) / 64;
      GramJob g;
      std::memset(&g, 0, sizeof(g));
      g.U = op_abs(P.factors[m]);
      g.wcol = op_ws(h.wcol);
      g.B = op_ws(h.gram);
      g.n = h.n;
      g.R = h.R;
      g.m = h.m;
      g.type = type;
      g.aat = h.aat ? 1 : 0;
      g.tiles = T * (T + 1) / 2;
      g.tile_begin = plan->gram_tiles;
      plan->gram_tiles += g.tiles;
      gjobs.push_back(g);
      const double kc = h.aat ? (double)h.R : (double)h.n;
      plan->flops += 2.0 * kc * 0.5 * h.m * (h.m + 1.0) + 4.0 / 3.0 * std::pow((double)h.m, 3.0);
      plan->gram_flops += 2.0 * kc * 0.5 * h.m * (h.m + 1.0);
      plan->mats.push_back(h);
    }
    plan->order.push_back(d);
  }
  // eigenvalues in the workspace when the caller passes no eigenvalue buffer
  plan->ws_ev = alloc(sizeof(double) * (size_t)plan->eval_elems);
  plan->ws_bytes = ws;
  // largest matrices first: the tridiagonalization CTAs run longest
  std::vector<int> idx(plan->mats.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return plan->mats[a].m > plan->mats[b].m; });
  std::vector<SubrankJob> sjobs;
  for (int i : idx) {
    const MatHost& h = plan->mats[i];
    SubrankJob s;
    std::memset(&s, 0, sizeof(s));
    s.B = op_ws(h.gram);
    s.d = op_ws(h.d);
    s.e = op_ws(h.e);
    s.ev = op_base(B_EVALS, sizeof(double) * h.ev_off);
    s.rank = op_base(B_SRANK, sizeof(int32_t) * (h.p * TKS_MAX_ORDER + h.mode));
    s.ell = op_base(B_ELL, sizeof(int32_t) * (h.p * TKS_MAX_ORDER + h.mode));
    s.m = h.m;
    s.order = plan->order[h.p];
    s.p = problems[h.p].oversampling[h.mode];
    s.eps = prm.trunc_tol;
    sjobs.push_back(s);
    plan->job_m.push_back(h.m);
  }
  plan->nw = (int)wjobs.size();
  plan->ng = (int)gjobs.size();
  plan->ns = (int)sjobs.size();
  std::vector<char> host;
  auto add = [&](const void* src, size_t bytes) {
    const size_t off = align_up(host.size(), 64);
    host.resize(off + bytes);
    std::memcpy(host.data() + off, src, bytes);
    return off;
  };
  plan->off_w = add(wjobs.data(), sizeof(WeightJob) * wjobs.size());
  plan->off_g = add(gjobs.data(), sizeof(GramJob) * gjobs.size());
  plan->off_s = add(sjobs.data(), sizeof(SubrankJob) * sjobs.size());
  const Status zero{0, 0};
  const size_t off_status = add(&zero, sizeof(zero));
  const std::vector<int32_t> zsteps(std::max<size_t>(1, sjobs.size()), 0);
  const size_t off_steps = add(zsteps.data(), sizeof(int32_t) * zsteps.size());
  cudaError_t e = cudaMalloc(&plan->arena, host.size());
  if (e != cudaSuccess) return reject(TKS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  // every tridiagonalization job records its executed steps in the arena
  plan->steps = reinterpret_cast<int32_t*>(plan->arena + off_steps);
  for (size_t i = 0; i < sjobs.size(); ++i)
    reinterpret_cast<SubrankJob*>(host.data() + plan->off_s)[i].steps = plan->steps + i;
  e = cudaMemcpy(plan->arena, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = prepare_subrank();
  if (e != cudaSuccess) {
    cudaFree(plan->arena);
    plan->arena = nullptr;
    return reject(TKS_ECUDA, std::string("subrank plan: ") + cudaGetErrorString(e));
  }
  plan->status = reinterpret_cast<Status*>(plan->arena + off_status);
  *out = plan;
  return TKS_OK;
}

void tks_subrank_plan_destroy(tks_subrank_plan* plan) {
  if (!plan) return;
  if (plan->arena) cudaFree(plan->arena);
  delete plan;
}

tks_status tks_subrank_info(const tks_subrank_plan* plan, tks_subrank_info_t* info) {
  if (!plan || !info) return fail(TKS_EINVAL, "null plan or info");
  std::memset(info, 0, sizeof(*info));
  info->workspace_bytes = plan->ws_bytes;
  info->eigenvalue_elems = plan->eval_elems;
  info->num_problems = plan->nprob;
  info->launches = 4;
  info->max_dim = plan->max_m;
  info->flops = plan->flops;
  return TKS_OK;
}

tks_status tks_subrank_executed_flops(const tks_subrank_plan* plan, double* flops) {
  if (!plan || !flops) return fail(TKS_EINVAL, "null plan or flops");
  std::vector<int32_t> st(plan->job_m.size(), 0);
  if (!st.empty())
    SR_CUDA_CHECK(cudaMemcpy(st.data(), plan->steps, sizeof(int32_t) * st.size(), cudaMemcpyDeviceToHost));
  double f = plan->gram_flops;
  for (size_t i = 0; i < st.size(); ++i) {
    const double m = plan->job_m[i];
    for (int k = 0; k < st[i]; ++k) f += 4.0 * (m - k) * (m - k);
  }
  *flops = f;
  return TKS_OK;
}

tks_status tks_subrank_problem_info(const tks_subrank_plan* plan, int32_t problem, int32_t* dims_out,
                                    int64_t* eig_off_out) {
  if (!plan || !dims_out || !eig_off_out) return fail(TKS_EINVAL, "null argument");
  if (problem < 0 || problem >= plan->nprob) return fail(TKS_EINVAL, "problem index out of range");
  for (int m = 0; m < TKS_MAX_ORDER; ++m) {
    dims_out[m] = 0;
    eig_off_out[m] = 0;
  }
  for (const MatHost& h : plan->mats)
    if (h.p == problem) {
      dims_out[h.mode] = h.m;
      eig_off_out[h.mode] = h.ev_off;
    }
  return TKS_OK;
}

tks_status tks_effective_subrank(tks_subrank_plan* plan, void* workspace, int32_t* ranks_out, int32_t* ell_out,
                                 double* eigenvalues_out, void* stream) {
  if (!plan) return fail(TKS_EINVAL, "null plan");
  if (!workspace || !ranks_out || !ell_out) return fail(TKS_EINVAL, "workspace, ranks_out and ell_out are required");
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0) return fail(TKS_EINVAL, "workspace not 256-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Bases b;
  std::memset(&b, 0, sizeof(b));
  char* w = static_cast<char*>(workspace);
  b.p[B_WS] = w;
  b.p[B_EVALS] = eigenvalues_out ? reinterpret_cast<char*>(eigenvalues_out) : w + plan->ws_ev;
  b.p[B_SRANK] = reinterpret_cast<char*>(ranks_out);
  b.p[B_ELL] = reinterpret_cast<char*>(ell_out);
  const auto* wj = reinterpret_cast<const WeightJob*>(plan->arena + plan->off_w);
  const auto* gj = reinterpret_cast<const GramJob*>(plan->arena + plan->off_g);
  const auto* sj = reinterpret_cast<const SubrankJob*>(plan->arena + plan->off_s);
  launch_subrank_weights(wj, plan->nw, b, s);
  launch_gram_f64(gj, plan->ng, plan->gram_tiles, b, s);
  launch_tridiag_f64(sj, plan->ns, plan->max_m, b, plan->status, s);
  launch_subrank_eig(sj, plan->ns, plan->max_m, b, plan->status, s);
  SR_CUDA_CHECK(cudaGetLastError());
  return TKS_OK;
}

tks_status tks_subrank_sync_status(tks_subrank_plan* plan, void* stream) {
  if (!plan) return fail(TKS_EINVAL, "null plan");
  SR_CUDA_CHECK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  Status h{0, 0};
  SR_CUDA_CHECK(cudaMemcpy(&h, plan->status, sizeof(h), cudaMemcpyDeviceToHost));
  if (h.code != 0) {
    const Status zero{0, 0};
    SR_CUDA_CHECK(cudaMemcpy(plan->status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    return fail(static_cast<tks_status>(h.code),
                std::string("device reported ") + tks_status_string(static_cast<tks_status>(h.code)));
  }
  return TKS_OK;
}

}  // extern "C"

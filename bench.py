#!/usr/bin/env python3
"""Throughput benchmark of the sketched Tucker-sum recompression on GB300.

A step is one tucker_sum_recompress call over a batch of P independent Tucker sums of the
decay512 shape (d=3, n=512, K=32 terms with ranks ~ U{8..32} per mode, Khatri-Rao sketch,
target rank 48, oversampling 10; seeded synthetic inputs already resident in HBM).  The
value is recompressions per second over all ranks.  Under torchrun every rank runs its own
batch on its own GPU (weak scaling, no data-path collective).

The default precision is TKS_MIXED: the contractions on tcgen05 tensor cores (bf16 operands,
float32 accumulation), the QR of each sketch and the ST-HOSVD in float64.

Also reported on the same JSON line:
  e2e           the same metric with the inputs copied from pinned host memory and the
                result read back inside every timed step
  roofline      the dominant launch: algorithmic flops (or bytes) per launch / its average
                CUDA-event duration inside the timed region, against the measured peak
  projection_tensor_roofline  the fused projection launch against the bf16 tensor peak
  cpu_baseline  the FP64 oracle timed on this host's cores on a bounded sample
  fp64_path     (mixed precision only) the plain FP64 GPU path on the same batch
  vs_oracle     sampled entries of the first recompressions against the FP64 oracle
  mixed_f32la   (precision mixed) the same batch with float32 QR and ST-HOSVD
  workloads     short runs of the other workloads (256-problem batch, order-4 Khatri-Rao and
                Kronecker): rate, FP64-path rate, speedup, error against the oracle
  subrank       the effective subrank heuristic (Alg. 5, float64) on the same batch: problems/s,
                its float64 roofline, and the oracle's rate on a sample
  backward      config 5: the backward of the sketch-and-project stage (Q fixed) over 152 grad384
                problems, mixed and float64 paths, their difference and the error against the
                oracle's gradient
  clocks        nvidia-smi SM clocks and throttle reasons sampled during the timed region

``--impl reference`` times the FP64 CPU oracle (the reference arm) instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Tucker-sum recompressions/s & TFLOP/s vs plain FP64 GPU path at ≤1e-5 rel err"
UNIT = "recompressions/s"
L2_BYTES = 129e6
# float64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA (4 flops) per clock x 2070 MHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed", "mixed_f32la"], default="mixed",
                    help="mixed: tensor-core contractions with float64 QR and ST-HOSVD (TKS_MIXED); mixed_f32la: "
                         "the same contractions with float32 QR and ST-HOSVD")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 comparison")
    ap.add_argument("--problems", type=int, default=None,
                    help="independent sums per step and GPU (default: 152; 256 for batched, 38 for order4)")
    ap.add_argument("--workload", default="decay512",
                    choices=["decay512", "order4-krp", "order4-kron", "batched", "exact_recovery"])
    ap.add_argument("--no-graph", action="store_true", help="time eager launches instead of graph replays")
    ap.add_argument("--seed", type=int, default=20260315)
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="budget of the cpu_baseline sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--measure-peaks", action="store_true", help="print FP64/FP32/TF32/BF16 GEMM rates")
    ap.add_argument("--lanes", type=int, default=None,
                    help="groups of problems whose recompressions run on concurrent streams (tks_params.lanes); "
                         "default: 2 for mixed_f32la on decay512 and batched, else 1 (with the float64 "
                         "ST-HOSVD every stage is throughput-bound and extra lanes measured slower)")
    ap.add_argument("--no-subrank", action="store_true", help="skip the effective subrank (Alg. 5) leg")
    ap.add_argument("--no-f32la", action="store_true", help="skip the float32-linear-algebra comparison leg")
    ap.add_argument("--oracle-problems", type=int, default=2,
                    help="problems whose recompression is checked against the FP64 oracle (sampled entries)")
    ap.add_argument("--extra-workloads", default="batched,order4-krp,order4-kron",
                    help="comma list of other workloads timed briefly (mixed vs FP64 path, error vs oracle); "
                         "'' for none")
    ap.add_argument("--extra-steps", type=int, default=5, help="timed steps of each extra workload (mixed)")
    ap.add_argument("--subrank-eps", type=float, default=1e-6, help="tolerance of the Alg. 5 leg")
    ap.add_argument("--subrank-steps", type=int, default=3, help="timed calls of the Alg. 5 leg")
    ap.add_argument("--no-backward", action="store_true", help="skip the backward (config 5) leg")
    ap.add_argument("--no-autotune", action="store_true", help="run the built-in schedule rules untuned")
    ap.add_argument("--schedule", default=None,
                    help='fixed schedule knobs for the main plan as JSON, e.g. \'{"sketch_qr": 3, "hosvd_r": 3}\' '
                         "(no autotuning; for profiling the tuned launch sequence without the search)")
    ap.add_argument("--backward-problems", type=int, default=152, help="grad384 problems per backward call")
    ap.add_argument("--backward-steps", type=int, default=20, help="timed calls of the mixed backward")
    args = ap.parse_args()
    if args.problems is None:
        args.problems = EXTRA_PROBLEMS.get(args.workload, 152)
    return args


WORKLOAD_LABELS = {
    "decay512": "decay512 x{P}: d=3, n=512, K=32, r~U{{8..32}}, mode spectra 10^(-i/8), Khatri-Rao, target 48, "
                "oversampling 10",
    "order4-krp": "order4 x{P}: d=4, n=256, K=64, r~U{{4..24}}, cores N(0,1) 2^(-k/4), Khatri-Rao, target 40, "
                  "oversampling 8",
    "order4-kron": "order4 x{P}: d=4, n=256, K=64, r~U{{4..24}}, cores N(0,1) 2^(-k/4), Kronecker, target 40, "
                   "oversampling 8",
    "batched": "batched: {P} sums, d=3, n~U{{128,256,512,1024}}, K~U{{8..48}}, r~U{{4..32}}, Khatri-Rao, "
               "target 1.5 x median rank, oversampling 5",
    "exact_recovery": "exact_recovery x{P}: d=3, n=64, K=4, r=8, Kronecker, target 32",
}


def workload_label(P, workload="decay512"):
    return WORKLOAD_LABELS[workload].format(P=P)


def workload_kind(workload):
    return "kron" if workload in ("order4-kron", "exact_recovery") else "krp"


def sampled_entries(core, factors, idx):
    """Entries of the Tucker tensor [[core; factors]] at integer index rows idx (m x d)."""
    import numpy as np
    W = np.einsum("ia,ib,ic,abc->i", factors[0][idx[:, 0]], factors[1][idx[:, 1]], factors[2][idx[:, 2]], core) \
        if core.ndim == 3 else None
    if W is None:
        out = []
        for ii in idx:
            T = core
            for k, U in enumerate(factors):
                T = np.tensordot(U[ii[k]], T, axes=(0, 0))
            out.append(float(T))
        W = np.array(out)
    return W


def problem_seeds(P, seed, rank):
    """Seeds of the P problems of one rank: disjoint across ranks (weak scaling)."""
    return [seed + 7919 * (rank * P + i) for i in range(P)]


def make_problems(P, seed, rank, bf16, workload="decay512"):
    from paper_2603_13532_gb300 import workloads as wl
    if workload == "batched":
        return wl.batched(seed=seed + 7919 * rank, num_problems=P, bf16=bf16).problems
    probs = []
    for s in problem_seeds(P, seed, rank):
        if workload == "decay512":
            probs += wl.decay512(seed=s, bf16=bf16).problems
        elif workload.startswith("order4"):
            probs += wl.order4(seed=s, kind=workload_kind(workload), bf16=bf16).problems
        else:
            probs += wl.exact_recovery(seed=s).problems
    return probs


def max_over_ranks(x, device):
    """The maximum of a per-rank float over all ranks of the default process group (x if none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(P, world, steps, elapsed_max):
    """Whole-job throughput: every rank processed P problems per step; time = slowest rank."""
    return P * world * steps / elapsed_max


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return dict(FALLBACK), "fallback"


# ------------------------------------------------------------------ clocks
CLOCK_FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + ",".join(CLOCK_FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self, gpu_index):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) == len(CLOCK_FIELDS):
                    rows.append(parts)
        os.unlink(self.path)
        idxs = sorted({r[0] for r in rows})
        pick = idxs[0] if len(idxs) == 1 else str(gpu_index)
        rows = [r for r in rows if r[0] == pick]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ------------------------------------------------------------------ CPU oracle
def oracle_rate(problems, seed0, budget_s, kind, rounding):
    """Recompressions/s of the FP64 oracle over as many problems as fit in budget_s."""
    from oracle import sketch_sum as ss
    done, t0 = 0, time.perf_counter()
    for i, p in enumerate(problems):
        ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=seed0, problem=i, rounding=rounding,
                      alpha=p.alpha)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def oracle_rate_one_core(workload, seed, bf16, count=2):
    """The oracle's rate with BLAS and OpenMP pinned to one thread, in a child process (the thread
    counts are fixed when numpy loads), on the first `count` problems of the same batch."""
    code = ("import json, sys, time; sys.path.insert(0, %r); import bench; "
            "p = bench.make_problems(%d, %d, 0, %r, %r); "
            "r, n, dt = bench.oracle_rate(p, %d, 1e9, bench.workload_kind(%r), %r); "
            "print(json.dumps([r, n, dt]))") % (ROOT, count, seed, bf16, workload, seed, workload,
                                                "bf16" if bf16 else None)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        rate, done, dt = json.loads(out.stdout.strip().splitlines()[-1])
        return {"value": rate, "cores": 1, "sample": f"{done} problems in {dt:.1f} s, one BLAS/OpenMP thread"}
    except Exception as e:   # the baseline is informative only
        return {"value": None, "cores": 1, "sample": f"not measured: {type(e).__name__}"}


def oracle_subrank_rate(problems, eps, budget_s):
    """Problems/s of the FP64 oracle's effective subrank heuristic over a bounded sample."""
    from oracle import subrank as sr
    done, t0 = 0, time.perf_counter()
    for p in problems:
        sr.effective_subrank(p.terms(), eps, p.oversampling, alpha=p.alpha)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def run_reference(args, rank, world):
    import torch.distributed as dist
    if rank != 0:
        return
    from paper_2603_13532_gb300 import workloads as wl
    bf16 = args.precision != "fp64" and args.workload != "exact_recovery"
    per_step = 2
    kind = workload_kind(args.workload)
    probs = make_problems(per_step * (args.steps + args.warmup), args.seed, 0, bf16, args.workload)
    rounding = "bf16" if bf16 else None
    from oracle import sketch_sum as ss
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for i in range(per_step):
            p = probs[s * per_step + i]
            ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=args.seed, problem=i, rounding=rounding,
                          alpha=p.alpha)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * len(times) / total
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_label(per_step, args.workload) + " (reference arm: float64 CPU oracle)",
                       "problems_per_step": per_step, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} problems per step, {args.steps} timed steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    del wl, dist


# ------------------------------------------------------------------ GPU arm
def time_steps(fn, steps, stream):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / 1e3


def graph_step(plan, out, ranks, stream, use_graph=True):
    """The plan's recompression into (out, ranks) as a callable: a CUDA-graph replay of the whole
    launch sequence (or an eager call).  Runs it once, synchronized, before returning."""
    import torch
    step = lambda: plan.recompress_raw(out, ranks)
    step()
    plan.sync()
    if not use_graph:
        return step, None
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()
    stream.wait_stream(side)
    with torch.cuda.graph(graph):
        step()
    graph.replay()
    torch.cuda.synchronize()
    return graph.replay, graph


def _rms(x):
    import numpy as np
    return float(np.sqrt(np.mean(np.asarray(x) ** 2)))


def oracle_errors(results, problems, kind, seed, rounding, count, nsamp=256):
    """The first `count` recompressions of a batch against the FP64 oracle on the same Gaussian draws,
    on nsamp sampled entries per problem: rel_err = rms(x_gpu - x_oracle) / rms(x_oracle) and
    trunc_diff = |rms(x_gpu - x) - rms(x_oracle - x)| / rms(x), x the sum evaluated term by term."""
    import numpy as np
    from oracle import sketch_sum as ss
    worst_rel = worst_tr = 0.0
    ranks_ok = True
    count = min(count, len(problems))
    for i in range(count):
        p = problems[i]
        ref = ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=seed, problem=i, rounding=rounding,
                            alpha=p.alpha)
        g = np.random.default_rng(1000 + i)
        idx = np.stack([g.integers(0, n, size=nsamp) for n in p.dims], axis=1)
        eg = sampled_entries(results[i]["core"], results[i]["factors"], idx)
        eo = sampled_entries(ref["core"], ref["factors"], idx)
        alpha = p.alpha if p.alpha is not None else [1.0] * p.num_terms
        ex = sum(a * sampled_entries(G, Us, idx) for a, (G, Us) in zip(alpha, p.terms()))
        worst_rel = max(worst_rel, _rms(eg - eo) / _rms(eo))
        worst_tr = max(worst_tr, abs(_rms(eg - ex) - _rms(eo - ex)) / _rms(ex))
        ranks_ok = ranks_ok and list(results[i]["ranks"]) == list(ref["ranks"])
    return {"rel_err": worst_rel, "trunc_err_diff": worst_tr, "ranks_match": ranks_ok, "problems": count,
            "samples_per_problem": nsamp,
            "note": "max over the first problems of the batch: rms difference of sampled entries of the "
                    "recompressed tensor from the FP64 oracle's (same Gaussian draws), relative to the oracle "
                    "entries' rms; and the difference of the two truncation errors relative to rms(X)"}


EXTRA_PROBLEMS = {"batched": 256, "order4-krp": 38, "order4-kron": 38}


def extra_workload_leg(args, workload, device, stream, rank, world):
    """A short measurement of another workload: the mixed path (graph replays), the plain FP64 path
    on the same inputs and Gaussian draws, and the error against the FP64 oracle."""
    import torch
    from paper_2603_13532_gb300 import binding
    P = EXTRA_PROBLEMS[workload]
    kind = workload_kind(workload)
    lanes = 2 if (args.precision == "mixed_f32la" and not workload.startswith("order4")) else 1
    problems = make_problems(P, args.seed, rank, True, workload)
    plan = binding.Plan(problems, kind=kind, precision=args.precision, seed=args.seed, device=device, lanes=lanes,
                        autotune=not args.no_autotune)
    tuning = plan.tuning()
    out = torch.zeros(plan.info.output_elems, dtype=torch.float64, device=device)
    ranks_t = torch.zeros(P * binding.MAX_ORDER, dtype=torch.int32, device=device)
    timed, graph = graph_step(plan, out, ranks_t, stream)
    el = max_over_ranks(time_steps(timed, args.extra_steps, stream), device)
    plan.sync()
    value = weak_scaling_rate(P, world, args.extra_steps, el)
    res = plan.unpack(out, ranks_t)
    leg = {"workload": workload_label(P, workload), "precision": args.precision, "value": value, "unit": UNIT,
           "ms_per_step": 1e3 * el / args.extra_steps, "steps": args.extra_steps, "lanes": tuning["picked"]["lanes"],
           "schedule": {"knobs": tuning["picked"], "autotuned": bool(tuning["autotuned"]),
                        "gain": (tuning["rule_ms"] / tuning["picked_ms"]) if tuning["autotuned"] else None},
           "tflops": (plan.info.flops_lowprec + plan.info.flops_fp64) * world * args.extra_steps / el / 1e12}
    del graph, plan
    plan64 = binding.Plan(problems, kind=kind, precision="fp64", seed=args.seed, device=device, omega_lowprec=True)
    out64 = torch.zeros(plan64.info.output_elems, dtype=torch.float64, device=device)
    r64 = torch.zeros_like(ranks_t)
    step64 = lambda: plan64.recompress_raw(out64, r64)
    step64()
    plan64.sync()
    steps64 = 1 if workload.startswith("order4") else 2
    el64 = max_over_ranks(time_steps(step64, steps64, stream), device)
    plan64.sync()
    v64 = weak_scaling_rate(P, world, steps64, el64)
    leg["fp64_path"] = {"value": v64, "unit": UNIT, "ms_per_step": 1e3 * el64 / steps64, "steps": steps64}
    leg["speedup"] = value / v64
    del plan64
    if rank == 0:
        leg["vs_oracle"] = oracle_errors(res, problems, kind, args.seed, "bf16",
                                         1 if workload.startswith("order4") else 2)
    return leg


def backward_leg(args, device, stream, rank, world):
    """Config 5 (grad384: d=3, n=384, K=16 terms of rank 16, bf16 inputs, target 32 + 8): the backward
    of the sketch-and-project stage with Q fixed over a batch of P such problems, on the mixed path
    (tensor-core products, float32 accumulation) and on the float64 path, with Q and Hbar resident on
    the device; plus the difference between the two and the error of the first problem against the
    oracle's float64 gradient."""
    import numpy as np
    import torch
    from paper_2603_13532_gb300 import binding, workloads as wl
    from oracle import sketch_sum as ss
    P = args.backward_problems
    problems = [wl.grad384(seed=20260318 + 1000 * rank + i).problems[0] for i in range(P)]
    g = np.random.default_rng(args.seed + 7 * rank)
    Qs = [[np.linalg.qr(g.standard_normal((p.dims[m], p.target[m] + p.oversampling[m])))[0] for m in range(3)]
          for p in problems]
    Hbars = [g.standard_normal([p.target[m] + p.oversampling[m] for m in range(3)]) for p in problems]
    res = {}
    grads = {}
    for prec in ("mixed", "fp64"):
        plan = binding.Plan(problems, kind="krp", precision=prec, seed=args.seed, device=device)
        Q = plan.pack_bases(Qs)
        Hb = plan.pack_core(Hbars)
        dc = torch.zeros(max(1, plan.info.grad_core_elems), dtype=torch.float64, device=device)
        df = torch.zeros(max(1, plan.info.grad_factor_elems), dtype=torch.float64, device=device)
        call = lambda: plan.backward_raw(Q, Hb, dc, df)
        for _ in range(args.warmup):
            call()
        plan.sync()
        steps = args.backward_steps if prec == "mixed" else max(1, args.backward_steps // 5)
        el = max_over_ranks(time_steps(call, steps, stream), device)
        plan.sync()
        res[prec] = {"value": weak_scaling_rate(P, world, steps, el), "unit": "gradients/s",
                     "ms_per_call": 1e3 * el / steps, "steps": steps}
        grads[prec] = (dc.clone(), df.clone())
        res[prec]["gpu_launches_per_call"] = int(plan.info.launches_backward)
        del plan
    def rel(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    leg = {"workload": f"grad384 x{P} (d=3, n=384, K=16, rank 16, bf16 inputs, b=40)",
           "value": res["mixed"]["value"], "unit": "gradients/s", "ms_per_call": res["mixed"]["ms_per_call"],
           "steps": res["mixed"]["steps"], "gpu_launches_per_call": res["mixed"]["gpu_launches_per_call"],
           "fp64_path": res["fp64"], "speedup": res["mixed"]["value"] / res["fp64"]["value"],
           "rel_diff_vs_fp64": {"dcores": rel(grads["mixed"][0], grads["fp64"][0]),
                                "dfactors": rel(grads["mixed"][1], grads["fp64"][1])},
           "timing": "eager launches of tks_project_core_backward with Q, Hbar and the outputs on the device"}
    if rank == 0:
        p = problems[0]
        rG, rU = ss.project_core_vjp(p.terms(), Qs[0], Hbars[0])
        dc = grads["mixed"][0].cpu().numpy()
        df = grads["mixed"][1].cpu().numpy()
        nc = sum(G.size for G in p.cores)
        ref_c = np.concatenate([G.ravel(order="F") for G in rG])
        R = [sum(G.shape[m] for G in p.cores) for m in range(3)]
        off, errs = 0, []
        for m in range(3):
            ref_f = np.hstack([rU[k][m] for k in range(p.num_terms)]).ravel(order="F")
            errs.append(np.linalg.norm(df[off: off + ref_f.size] - ref_f) / np.linalg.norm(ref_f))
            off += p.dims[m] * R[m]
        if not args.no_cpu:
            t0, done = time.perf_counter(), 0
            while done < P and time.perf_counter() - t0 < args.cpu_seconds / 2:
                q = problems[done]
                ss.project_core_vjp(q.terms(), Qs[done], Hbars[done])
                done += 1
            dt = time.perf_counter() - t0
            leg["cpu_baseline"] = {"value": done / dt, "unit": "gradients/s", "cores": os.cpu_count(),
                                   "kind": "oracle",
                                   "sample": f"{done} of the {P} problems in {dt:.1f} s (numpy float64 "
                                             f"vector-Jacobian product, BLAS on all host cores)"}
        leg["vs_oracle"] = {"dcores": float(np.linalg.norm(dc[:nc] - ref_c) / np.linalg.norm(ref_c)),
                            "dfactors": float(max(errs)), "problems": 1,
                            "note": "relative Frobenius error of the first problem's mixed gradients against "
                                    "the oracle's float64 vector-Jacobian product"}
    return leg


FP32_PEAK_TFLOPS = 152 * 256 * 2.070e9 / 1e12   # 128 FP32 FMA per SM per clock
FP64_KINDS = {"gemm", "reduce", "qr", "core_sketch", "tsqr64", "svd64", "ttm64", "chol"}
TENSOR_FP64_KINDS = {"oz_gemm", "oz_gram"}
FP32_KINDS = {"simt", "core_sketch32", "qr32", "svd32", "tsqr32", "core_sketch3", "chain3", "qr_smem32",
              "project3", "sketch3", "qr_reg32", "ttm32", "fold4", "project4", "sketch3f", "sketch4"}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch per problem, from an ncu
# capture of the same kernel binary on 16 decay512 problems (15.594 MB read + 0.274 MB written),
# used to scale the measured traffic to the bench launch; only valid for that kernel and workload.
NCU_TRAFFIC_PER_PROBLEM = {("decay512", "project3"): (15.593984e6 + 0.273920e6) / 16}


def project3_tensor_flops(plan, problems):
    """Algorithmic flops of the fused projection's tensor-core contraction (s3: 2 b0 b1 b2 r_k3 per
    term) over the problems that take that kernel (order 3, b2, b3 <= 64, mixed precision)."""
    total = 0.0
    for p, pi in zip(problems, plan.pinfo):
        b = [pi.basis_cols[m] for m in range(p.order)]
        if p.order != 3 or b[1] > 64 or b[2] > 64:
            continue
        total += sum(2.0 * b[0] * b[1] * b[2] * r[2] for r in p.ranks())
    return total


def roofline_from_profile(prof, calls, peaks, workload=None, problems=0, tensor_flops=None):
    """The longest launch with an algorithmic count, and its achieved rate against its roofline.

    FP64 CUDA-core launches are bound by the FP64 pipe, FP32 CUDA-core launches by the FP32 pipe
    (peaks from unit counts and the 2070 MHz clock); tensor-core launches by the tensor pipe or
    HBM, whichever the launch's algorithmic arithmetic intensity puts first (ridge = sustained
    bf16 peak / HBM bandwidth).  The fused projection runs on two pipes at once: its first two
    contractions on the FP32 pipe and the third (`tensor_flops`) on the tensor pipe as six bf16
    products of split operands; its peak is the rate at which the busier of the two pipes would
    finish the launch's algorithmic flops.
    """
    total_ms = sum(s["ms"] for s in prof)
    # the dominant kernel: the launch kind with the largest share of the step among those with an
    # algorithmic count, its launches taken together (flops and time summed)
    groups = {}
    for s_ in prof:
        if s_["flops"] > 0 or s_["bytes"] > 0:
            g = groups.setdefault(s_["kind"], {"kind": s_["kind"], "ms": 0.0, "flops": 0.0, "bytes": 0.0,
                                               "launches": 0, "names": []})
            g["ms"] += s_["ms"]
            g["flops"] += s_["flops"]
            g["bytes"] += s_["bytes"]
            g["launches"] += 1
            g["names"].append(s_["name"])
    top = max(groups.values(), key=lambda g: g["ms"]) if groups else dict(max(prof, key=lambda s_: s_["ms"]),
                                                                          launches=1, names=[])
    if not top["names"]:
        top["names"] = [top.get("name", "")]
    top["name"] = top["names"][0] if top["launches"] == 1 else f'{top["kind"]} ({top["launches"]} launches)'
    overall_top = max(prof, key=lambda s_: s_["ms"])
    # per launch: the group's flops and time divided by its launches
    top["flops"] /= top["launches"]
    top["bytes"] /= top["launches"]
    avg_s = top["ms"] / 1e3 / max(1, calls) / top["launches"]
    kind = top["kind"]
    if kind == "project3" and top["flops"] > 0 and tensor_flops:
        f_tc = min(tensor_flops, top["flops"])
        t_alu = (top["flops"] - f_tc) / (FP32_PEAK_TFLOPS * 1e12)
        t_tc = 6.0 * f_tc / (peaks["bf16_tflops_sustained"] * 1e12)
        roof = {"bound": "alu" if t_alu >= t_tc else "tensor", "achieved": top["flops"] / avg_s / 1e12,
                "peak": top["flops"] / max(t_alu, t_tc) / 1e12, "unit": "TFLOP/s",
                "peak_source": "two pipes: s1, s2 on the FP32 pipe (derived 152 SMs x 256 flop/clk x 2070 MHz), "
                               "s3 as 6 bf16 products on the tensor pipe (measured bf16 sustained / 6); peak = "
                               "algorithmic flops / the longer of the two pipe times",
                "tensor_flops_per_launch": f_tc}
    elif kind in FP64_KINDS and top["flops"] > 0:
        roof = {"bound": "alu", "achieved": top["flops"] / avg_s / 1e12, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "derived FP64: 152 SMs x 4 flop/clk x 2070 MHz"}
    elif kind in FP32_KINDS and top["flops"] > 0:
        roof = {"bound": "alu", "achieved": top["flops"] / avg_s / 1e12, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "peak_source": "derived FP32: 152 SMs x 256 flop/clk x 2070 MHz"}
    else:
        ridge = peaks["bf16_tflops_sustained"] * 1e12 / (peaks["hbm_gbs"] * 1e9)
        ai = top["flops"] / top["bytes"] if top["bytes"] > 0 else float("inf")
        if ai > ridge:
            roof = {"bound": "tensor", "achieved": top["flops"] / avg_s / 1e12,
                    "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                    "peak_source": "measured bf16 sustained"}
        else:
            roof = {"bound": "hbm", "achieved": top["bytes"] / avg_s / 1e9, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "peak_source": "measured hbm_gbs"}
        roof["arithmetic_intensity"] = ai
    roof["frac"] = roof["achieved"] / roof["peak"]
    per_problem = NCU_TRAFFIC_PER_PROBLEM.get((workload, kind))
    roof["traffic"] = per_problem * problems if per_problem is not None else None
    if per_problem is not None:
        roof["traffic_note"] = "ncu DRAM bytes of the kernel on 16 problems, scaled to this launch's problems"
    roof["kernel"] = top["name"]
    roof["launches_per_step"] = top["launches"]
    roof["kernel_share"] = top["ms"] / total_ms if total_ms > 0 else None
    roof["avg_launch_ms"] = avg_s * 1e3
    roof["algorithmic_flops_per_launch"] = top["flops"]
    roof["algorithmic_bytes_per_launch"] = top["bytes"]
    if overall_top["name"] not in top["names"]:
        roof["longest_launch"] = {"name": overall_top["name"],
                                  "share": overall_top["ms"] / total_ms if total_ms > 0 else None}
    return roof


def projection_tensor_roofline(prof, calls, peaks):
    """The fused projection launches (a7+a8) against the measured bf16 tensor peak (burst): their
    algorithmic flops per launch over their average CUDA-event duration."""
    rows = [s for s in prof if s["kind"] in ("project3", "project4") and s["flops"] > 0]
    if not rows:
        return None
    out = []
    for s in rows:
        avg = s["ms"] / 1e3 / max(1, calls)
        ach = s["flops"] / avg / 1e12
        out.append({"kernel": s["name"], "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": ach / peaks["bf16_tflops"], "avg_launch_ms": avg * 1e3,
                    "algorithmic_flops_per_launch": s["flops"], "peak_source": "measured bf16 burst"})
    return out


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.measure_peaks:
        measure_peaks()
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo" if args.impl == "reference" else "nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_2603_13532_gb300 import binding

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    bf16 = args.precision != "fp64"
    P = args.problems
    kind = workload_kind(args.workload)
    if args.workload == "exact_recovery" and args.precision != "fp64":
        raise SystemExit("the exact_recovery workload is float64 only")
    if args.lanes is None:
        args.lanes = 2 if (args.precision == "mixed_f32la" and not args.workload.startswith("order4")) else 1
    problems = make_problems(P, args.seed, rank, bf16, args.workload)
    fixed = json.loads(args.schedule) if args.schedule else None
    autotune = args.precision != "fp64" and not args.no_autotune and fixed is None
    t_tune = time.perf_counter()
    plan = binding.Plan(problems, kind=kind, precision=args.precision, seed=args.seed, device=device,
                        lanes=args.lanes, autotune=autotune, schedule=fixed)
    t_tune = time.perf_counter() - t_tune
    tuning = plan.tuning()
    schedule = {"knobs": tuning["picked"], "rule": tuning["rule"], "autotuned": bool(tuning["autotuned"])}
    if tuning["autotuned"]:
        schedule.update({"rule_ms": tuning["rule_ms"], "picked_ms": tuning["picked_ms"],
                         "gain": tuning["rule_ms"] / tuning["picked_ms"], "candidates": len(tuning["candidates"]),
                         "plan_create_s": t_tune,
                         "note": "greedy search in tks_plan_create from the built-in rules (lanes, sketch QR, "
                                 "ST-HOSVD factor, projection chunk, tensor-core stages), median of 3 eager "
                                 "recompressions per candidate"})
    out = torch.zeros(plan.info.output_elems, dtype=torch.float64, device=device)
    ranks_t = torch.zeros(P * binding.MAX_ORDER, dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream()

    def step():
        plan.recompress_raw(out, ranks_t)

    for _ in range(args.warmup):
        step()
    plan.sync()
    # per-stage times: CUDA events between the plan's launches over an eager pass of K steps
    plan.profile_begin(args.steps)
    eager_elapsed = time_steps(step, args.steps, stream)
    prof = plan.profile_end()
    plan.sync()
    # the whole recompression as one CUDA graph (the launch sequence is fixed per plan)
    timed, graph = graph_step(plan, out, ranks_t, stream, use_graph=not args.no_graph)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    elapsed = time_steps(timed, args.steps, stream)
    clock_info = clocks.stop(local)
    plan.sync()
    elapsed = max_over_ranks(elapsed, device)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ms_per_step = 1e3 * elapsed / args.steps
    value = weak_scaling_rate(P, world, args.steps, elapsed)
    tflops = (plan.info.flops_lowprec + plan.info.flops_fp64) * world * args.steps / elapsed / 1e12

    peaks, peak_src = load_peaks()
    roof = roofline_from_profile(prof, args.steps, peaks, args.workload, P,
                                 tensor_flops=project3_tensor_flops(plan, problems) if bf16 else None)
    roof["peak_file"] = peak_src

    # end to end: every step copies its inputs from pinned host memory, recompresses and reads the
    # result back to pinned host memory.  Two plans own two device input buffers, so step i's
    # copies (copy stream) overlap step i-1's recompression (compute stream); a buffer is refilled
    # only after the recompression that read it, and a result is read only after it is written.
    e2e = None
    if not args.no_e2e:
        host_in, _ = binding.pack_inputs(problems, plan.dtype, "cpu", pin=True)
        lanes = [(plan, out, ranks_t, timed)]
        plan_b = binding.Plan(problems, kind=kind, precision=args.precision, seed=args.seed, device=device,
                              schedule=tuning["picked"])
        out_b = torch.zeros_like(out)
        ranks_b = torch.zeros_like(ranks_t)
        plan_b.recompress_raw(out_b, ranks_b)
        plan_b.sync()
        timed_b = lambda: plan_b.recompress_raw(out_b, ranks_b)
        if graph is not None:
            graph_b = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                timed_b()
            stream.wait_stream(side)
            with torch.cuda.graph(graph_b):
                timed_b()
            timed_b = graph_b.replay
        lanes.append((plan_b, out_b, ranks_b, timed_b))
        host_out = [torch.empty_like(out, device="cpu").pin_memory() for _ in lanes]
        host_ranks = [torch.empty_like(ranks_t, device="cpu").pin_memory() for _ in lanes]
        copy = torch.cuda.Stream()        # host -> device
        back = torch.cuda.Stream()        # device -> host (the other copy direction runs alongside)
        done = [torch.cuda.Event() for _ in lanes]
        read = [torch.cuda.Event() for _ in lanes]
        for ev in done + read:
            ev.record(stream)
        torch.cuda.synchronize()
        counter = [0]

        def e2e_step():
            i = counter[0] % 2
            counter[0] += 1
            pl, o, r, run = lanes[i]
            copy.wait_event(done[i])                      # the previous recompression of this buffer
            with torch.cuda.stream(copy):
                pl.flat_inputs.copy_(host_in, non_blocking=True)
            loaded = torch.cuda.Event()
            loaded.record(copy)
            stream.wait_event(loaded)
            stream.wait_event(read[i])                    # the previous result of this buffer is read
            run()
            done[i].record(stream)
            back.wait_event(done[i])
            with torch.cuda.stream(back):
                host_out[i].copy_(o, non_blocking=True)
                host_ranks[i].copy_(r, non_blocking=True)
            read[i].record(back)

        e2e_step()
        e2e_step()
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        copy.wait_stream(stream)
        back.wait_stream(stream)
        for _ in range(args.steps):
            e2e_step()
        stream.wait_stream(back)                         # the last results are on the host
        end.record(stream)
        end.synchronize()
        e_el = max_over_ranks(start.elapsed_time(end) / 1e3, device)
        plan_b.sync()
        e2e = {"value": weak_scaling_rate(P, world, args.steps, e_el), "unit": UNIT,
               "h2d_bytes_per_step": int(host_in.numel() * host_in.element_size()),
               "d2h_bytes_per_step": int(out.numel() * 8 + ranks_t.numel() * 4),
               "pipelining": "two input buffers (two plans); host-to-device and device-to-host copies on "
                             "two streams of their own overlap the other buffer's recompression"}
        del plan_b

    # the plain FP64 GPU path on the same batch (same values, float64 storage), and the
    # difference of the two results on sampled entries of the recompressed tensors
    fp64_path = None
    if args.precision != "fp64" and args.fp64_steps > 0:
        import numpy as _np
        # the same Gaussian draws as the mixed plan, so the comparison below is arithmetic only
        plan64 = binding.Plan(problems, kind=kind, precision="fp64", seed=args.seed, device=device,
                              omega_lowprec=True)
        out64 = torch.zeros(plan64.info.output_elems, dtype=torch.float64, device=device)
        r64 = torch.zeros_like(ranks_t)

        def step64():
            plan64.recompress_raw(out64, r64)

        step64()
        plan64.sync()
        el64 = time_steps(step64, args.fp64_steps, stream)
        plan64.sync()
        res_m = plan.unpack(out, ranks_t)
        res_d = plan64.unpack(out64, r64)
        g = _np.random.default_rng(0)
        worst = worst_trunc = 0.0
        for pm, pd, pr in list(zip(res_m, res_d, problems))[:8]:
            idx = _np.stack([g.integers(0, n, size=256) for n in pr.dims], axis=1)
            em = sampled_entries(pm["core"], pm["factors"], idx)
            ed = sampled_entries(pd["core"], pd["factors"], idx)
            # the sum itself at the same entries, term by term
            alpha = pr.alpha if pr.alpha is not None else [1.0] * pr.num_terms
            ex = sum(a * sampled_entries(G, Us, idx) for a, (G, Us) in zip(alpha, pr.terms()))
            scale = float(_np.sqrt(_np.mean(ex ** 2)))
            worst = max(worst, float(_np.sqrt(_np.mean((em - ed) ** 2)) / _np.sqrt(_np.mean(ed ** 2))))
            trunc_m = float(_np.sqrt(_np.mean((em - ex) ** 2)))
            trunc_d = float(_np.sqrt(_np.mean((ed - ex) ** 2)))
            worst_trunc = max(worst_trunc, abs(trunc_m - trunc_d) / scale)
        v64 = P * args.fp64_steps / el64
        fp64_path = {"value": v64 * world, "unit": UNIT, "ms_per_step": 1e3 * el64 / args.fp64_steps,
                     "steps": args.fp64_steps, "speedup": value / (v64 * world),
                     "rel_diff_sampled": worst,
                     "rel_diff_note": "rms difference of 256 sampled entries per problem (8 problems) of the "
                                      "mixed and FP64 recompressed tensors (same Gaussian draws), relative to "
                                      "the FP64 entries' rms",
                     "trunc_err_diff_sampled": worst_trunc,
                     "trunc_err_note": "|e_mixed - e_fp64| / rms(X) with e = rms(X~ - X) over the same entries "
                                       "(X evaluated term by term): the accuracy target when the truncation is "
                                       "far from exact and the kept subspace is not unique"}
        del plan64

    # the same contractions with float32 QR and ST-HOSVD (TKS_MIXED_F32LA) on the same batch
    f32la = None
    if args.precision == "mixed" and not args.no_f32la:
        plan32 = binding.Plan(problems, kind=kind, precision="mixed_f32la", seed=args.seed, device=device,
                              lanes=1 if args.workload.startswith("order4") else 2, autotune=not args.no_autotune)
        out32 = torch.zeros(plan32.info.output_elems, dtype=torch.float64, device=device)
        r32 = torch.zeros_like(ranks_t)
        timed32, graph32 = graph_step(plan32, out32, r32, stream, use_graph=not args.no_graph)
        el32 = max_over_ranks(time_steps(timed32, args.steps, stream), device)
        plan32.sync()
        v32 = weak_scaling_rate(P, world, args.steps, el32)
        f32la = {"value": v32, "unit": UNIT, "ms_per_step": 1e3 * el32 / args.steps, "steps": args.steps,
                 "precision": "mixed_f32la", "schedule": plan32.tuning()["picked"],
                 "note": "the same tensor-core contractions with the QR of Y_n and the ST-HOSVD in float32 "
                         "(Householder QR, TSQR and one-sided Jacobi SVD; no Gram matrices)"}
        if fp64_path is not None:
            f32la["speedup_vs_fp64_path"] = v32 / fp64_path["value"]
        if rank == 0 and args.oracle_problems > 0:
            f32la["vs_oracle"] = oracle_errors(plan32.unpack(out32, r32), problems, kind, args.seed, "bf16",
                                               args.oracle_problems)
        del graph32, plan32

    # the effective subrank heuristic (Alg. 5) on the same batch and device inputs, float64
    subrank = None
    if not args.no_subrank:
        sp = binding.SubrankPlan(problems, args.subrank_eps, dtype=plan.dtype, device=device, inputs=plan.inputs)
        sr_rank = torch.zeros(P * binding.MAX_ORDER, dtype=torch.int32, device=device)
        sr_ell = torch.zeros_like(sr_rank)

        def run_subrank():
            sp.run_raw(sr_rank, sr_ell)

        run_subrank()
        sp.sync()
        el_sr = time_steps(run_subrank, args.subrank_steps, stream)
        sp.sync()
        el_sr = max_over_ranks(el_sr, device)
        got = sr_rank.cpu().numpy().reshape(-1, binding.MAX_ORDER)
        got = np.concatenate([got[i, :p.order] for i, p in enumerate(problems)])
        achieved = sp.info.flops * args.subrank_steps / el_sr / 1e12
        executed = sp.executed_flops()
        achieved_exec = executed * args.subrank_steps / el_sr / 1e12
        subrank = {"value": weak_scaling_rate(P, world, args.subrank_steps, el_sr), "unit": "problems/s",
                   "ms_per_call": 1e3 * el_sr / args.subrank_steps, "steps": args.subrank_steps,
                   "eps": args.subrank_eps, "launches_per_call": int(sp.info.launches),
                   "max_gram_order": int(sp.info.max_dim),
                   "ranks": {"min": int(got.min()), "mean": float(got.mean()), "max": int(got.max())},
                   "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                "frac": achieved / FP64_PEAK_TFLOPS,
                                "peak_source": "derived FP64: 152 SMs x 4 flop/clk x 2070 MHz",
                                "flops_per_call": sp.info.flops,
                                "flops_note": "Gram matrices 2 x contraction x m(m+1)/2 plus tridiagonalization "
                                              "4/3 m^3 per (problem, mode), m = min(n, R); the reduction "
                                              "ends early on numerically rank-deficient Gram matrices "
                                              "(decay512: after ~130 of 512 steps), so the count exceeds "
                                              "the executed work there",
                                "traffic": None,
                                "executed_flops_per_call": executed,
                                "achieved_executed": achieved_exec,
                                "frac_executed": achieved_exec / FP64_PEAK_TFLOPS,
                                "executed_note": "the Gram matrices plus 4 (m - k)^2 per reduction step the "
                                                 "tridiagonalization ran before its early end (read back from "
                                                 "the device after the calls)"}}
        if rank == 0 and not args.no_cpu:
            rate, done, dt = oracle_subrank_rate(problems, args.subrank_eps, args.cpu_seconds / 2)
            subrank["cpu_baseline"] = {"value": rate, "unit": "problems/s", "cores": os.cpu_count(),
                                       "kind": "oracle",
                                       "sample": f"{done} of the {P} problems in {dt:.1f} s (numpy eigvalsh of "
                                                 f"the R x R Gram matrices, LAPACK on all host cores)"}
        del sp

    backward = None
    if not args.no_backward and args.precision != "fp64":
        backward = backward_leg(args, device, stream, rank, world)

    extra = {}
    for wk in [w for w in args.extra_workloads.split(",") if w]:
        if wk == args.workload or args.precision == "fp64":
            continue
        extra[wk] = extra_workload_leg(args, wk, device, stream, rank, world)

    line = None
    if rank == 0:
        vs_oracle = None
        if args.oracle_problems > 0:
            vs_oracle = oracle_errors(plan.unpack(out, ranks_t), problems, kind, args.seed, "bf16" if bf16 else None,
                                      args.oracle_problems)
        in_bytes = plan.flat_inputs.numel() * plan.flat_inputs.element_size()
        cpu = None
        if not args.no_cpu:
            rate, done, dt = oracle_rate(problems, args.seed, args.cpu_seconds, kind,
                                         "bf16" if bf16 else None)
            cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"{done} of the {P} problems of this batch in {dt:.1f} s (numpy float64, "
                             f"BLAS on all host cores)",
                   "single_core": oracle_rate_one_core(args.workload, args.seed, bf16)}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "bf16",
                "data": "synthetic",
                "config": {"workload": workload_label(P, args.workload), "problems_per_step": P,
                           "precision": args.precision, "tflops": tflops,
                           "flops_per_step": plan.info.flops_lowprec + plan.info.flops_fp64,
                           "l2": f"inputs {in_bytes / 1e6:.0f} MB per GPU > L2 129 MB, no flush",
                           "parallelism": f"replicas x{world}",
                           "lanes": tuning["picked"]["lanes"] if args.precision != "fp64" else 1,
                           "schedule": schedule},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp64_path": fp64_path, "vs_oracle": vs_oracle,
                "mixed_f32la": f32la, "workloads": extra or None,
                "projection_tensor_roofline": projection_tensor_roofline(prof, args.steps, peaks),
                "subrank": subrank,
                "backward": backward,
                "gpu_launches": int(plan.info.launches_recompress) * args.steps,
                "timing": ("CUDA-graph replays of the whole recompression" if graph is not None
                           else "eager launches") + "; stage times from an eager pass with events (one "
                          "launch sequence: a profiled call does not split into lanes)",
                "eager_ms_per_step": 1e3 * eager_elapsed / args.steps,
                "clocks": clock_info,
                "stages": [{"name": s["name"], "ms_per_call": s["ms"] / max(1, s["calls"])} for s in prof]}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    del np


def measure_peaks():
    import torch
    dev = torch.device("cuda", 0)
    out = {}
    for name, dt, n, tf32 in [("fp64_tflops", torch.float64, 4096, False), ("fp32_tflops", torch.float32, 8192, False),
                              ("tf32_tflops", torch.float32, 8192, True), ("bf16_tflops", torch.bfloat16, 8192, False)]:
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device=dev, dtype=dt)
        b = torch.randn(n, n, device=dev, dtype=dt)
        for _ in range(3):
            a @ b
        torch.cuda.synchronize()
        best = 1e9
        for _ in range(5):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            a @ b
            e.record()
            e.synchronize()
            best = min(best, s.elapsed_time(e) / 1e3)
        out[name] = 2 * n ** 3 / best / 1e12
    print(json.dumps(out))


if __name__ == "__main__":
    main()

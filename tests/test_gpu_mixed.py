"""GPU parity of the mixed-precision path (TKS_MIXED) against the FP64 CPU oracle, through the C ABI.

The mixed path reads bfloat16 cores and factors and sketches with Omega drawn in float32 and
rounded to bfloat16 (oracle.rng.gaussian_f32); the oracle runs on the same bfloat16-valued inputs and the same rounded Omega in
float64, so every difference is arithmetic of the GPU path:

  Omega              bit-exact
  Y_n, H (given Q)   1e-5 relative Frobenius.  Products with bf16 inputs are exact in float32;
                     float32 operands enter the tensor cores as three bf16 planes (about 2^-24
                     relative) and every sum is accumulated in float32 (about 1e-7 relative per
                     element, times sqrt of the reduction length)
  recompression      |X~_gpu - X~_oracle| / ||X|| <= 1e-5 on sampled entries, and the two
                     truncation errors agree to 1e-5 (the accuracy target of the mixed path)
"""
import numpy as np
import pytest

from oracle import rng
from oracle import sketch_sum as ss
from oracle.tensor import tucker_entries, tucker_full, tucker_sum_full
from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


MODES = ["mixed", "mixed_f32la"]


def _plan(problems, kind, seed, tol=0.0, precision="mixed"):
    from paper_2603_13532_gb300 import binding
    return binding.Plan(problems, kind=kind, precision=precision, seed=seed, tol=tol)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _per_slice(a, b, tol, floor=1e-2):
    """Elementwise check beside the normwise one: along every axis, each slice (a column of Y, a
    mode-n slice of H) has max |a - b| within tol times its largest |b|, so an error confined to small
    entries or trailing rows cannot hide in the Frobenius norm.  A slice below floor times the largest
    |b| overall (a direction at the noise floor, e.g. beyond the sum's true rank, whose entries come
    from cancellation) is held to tol times that floor instead."""
    a, b = np.asarray(a), np.asarray(b)
    g = float(np.max(np.abs(b)))
    for axis in range(b.ndim):
        for k in range(b.shape[axis]):
            sa, sb = np.take(a, k, axis=axis), np.take(b, k, axis=axis)
            m = max(float(np.max(np.abs(sb))), floor * g)
            if m > 0:
                err = float(np.max(np.abs(sa - sb)))
                assert err <= tol * m, (axis, k, err / m)


def _bf16_problems(d, seed=0):
    """Ragged sizes: n a multiple of 8 (TMA row alignment) but not of the 128/64 tiles."""
    g = np.random.default_rng(200 + d + seed)
    probs = []
    for dims, K in ([[72, 40, 136, 48][:d], 3], [[24, 96, 8, 56][:d], 2], [[200] * d, 6]):
        cores, facs = [], []
        for _ in range(K):
            r = [min(int(x), n) for x, n in zip(g.integers(1, 9, size=d), dims)]
            cores.append(g.standard_normal(r))
            facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
        p = wl.Problem(list(dims), cores, facs, [6] * d, [2] * d, alpha=list(g.standard_normal(K)))
        probs.append(p)
    return wl._finish(probs, True)


def _oracle(p, kind, seed, problem, **kw):
    return ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=seed, problem=problem,
                         alpha=p.alpha, rounding="bf16", **kw)


def test_mixed_omega_is_rounded_draws(cuda_lib):
    probs = _bf16_problems(3)
    plan = _plan(probs, "krp", 31)
    om = plan.omega()
    for p, (prob, pi) in enumerate(zip(probs, plan.pinfo)):
        for m in range(3):
            ref = rng.omega(31, p, m, prob.dims[m], pi.omega_cols[m], rounding="bf16")
            assert np.array_equal(om[p][m], ref)


def test_mixed_omega_matches_golden_heads(cuda_lib):
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                       "omega_head.json")))
    for entry in gold["draws"]:
        p = entry["problem"]
        probs = wl._finish([wl.exact_recovery(n=16, K=1, r=2, target=2).problems[0] for _ in range(p + 1)],
                           True)
        for q in probs:
            q.target = [4, 4, 4]
            q.oversampling = [0, 0, 0]
        om = _plan(probs, "krp", entry["seed"]).omega()[p][entry["mode"]].ravel(order="F")[:32]
        want = np.array([float.fromhex(h) for h in entry["bf16_values"]])
        assert np.array_equal(om, want)


@pytest.mark.parametrize("kind", ["krp", "kron"])
def test_fp64_plan_with_the_mixed_draws_matches_the_oracle(cuda_lib, kind):
    """omega_lowprec: a float64 plan on the mixed modes' Omega equals the oracle's low-precision
    sketch to float64 accuracy (the bench compares the mixed and float64 paths this way)."""
    from paper_2603_13532_gb300 import binding
    probs = _bf16_problems(3, 4)
    plan = binding.Plan(probs, kind=kind, precision="fp64", seed=15, omega_lowprec=True)
    Ys = plan.sketch()
    for i, prob in enumerate(probs):
        ref = _oracle(prob, kind, 15, i)
        for m in range(3):
            assert _rel(Ys[i][m], ref["Y"][m]) <= 1e-12


@pytest.mark.parametrize("kind", ["krp", "kron"])
@pytest.mark.parametrize("d", [3, 4])
def test_mixed_sketch_matches_oracle(cuda_lib, kind, d):
    probs = _bf16_problems(d)
    Ys = _plan(probs, kind, 5).sketch()
    for i, prob in enumerate(probs):
        ref = _oracle(prob, kind, 5, i)
        for m in range(d):
            assert _rel(Ys[i][m], ref["Y"][m]) <= 1e-5, (kind, d, i, m, _rel(Ys[i][m], ref["Y"][m]))
            _per_slice(Ys[i][m], ref["Y"][m], 1e-5)


@pytest.mark.parametrize("kind", ["krp", "kron"])
@pytest.mark.parametrize("d", [2, 3, 4])
def test_mixed_projection_matches_oracle_given_q(cuda_lib, kind, d):
    probs = _bf16_problems(d, 1)
    refs = [_oracle(p, kind, 6, i) for i, p in enumerate(probs)]
    Hs = _plan(probs, kind, 6).project([r["Q"] for r in refs])
    for H, r in zip(Hs, refs):
        assert _rel(H, r["H"]) <= 1e-5
        _per_slice(H, r["H"], 1e-5)


def test_mixed_krp_sketch_order3_term_kernel_edges(cuda_lib):
    """Khatri-Rao sketches of order-3 terms at the edges of the per-term kernel: ranks 1, 3 (not a
    multiple of its 4-wide loads), 32 (its limit) and 33 (per-mode fallback) in one problem with
    s = 64 (its column limit), and a problem with s = 66 that takes the per-mode kernels."""
    g = np.random.default_rng(78)
    specs = [([64, 72, 80], [[1, 1, 1], [3, 5, 7], [32, 32, 32], [33, 9, 4], [12, 32, 30]], [56, 60, 50], [8, 4, 8]),
             ([72, 72, 72], [[6, 7, 8], [20, 3, 11]], [60, 60, 60], [6, 6, 6])]
    probs = []
    for dims, ranks, target, over in specs:
        cores = [g.standard_normal(r) for r in ranks]
        facs = [[g.standard_normal((n, ri)) for n, ri in zip(dims, r)] for r in ranks]
        probs.append(wl.Problem(dims, cores, facs, target, over, alpha=list(g.standard_normal(len(ranks)))))
    probs = wl._finish(probs, True)
    plan = _plan(probs, "krp", 9)
    assert [pi.sketch_cols[0] for pi in plan.pinfo] == [64, 66]
    Ys = plan.sketch()
    for i, prob in enumerate(probs):
        ref = _oracle(prob, "krp", 9, i)
        for m in range(3):
            assert _rel(Ys[i][m], ref["Y"][m]) <= 1e-5, (i, m, _rel(Ys[i][m], ref["Y"][m]))
            _per_slice(Ys[i][m], ref["Y"][m], 1e-5)


@pytest.mark.parametrize("kind", ["krp", "kron"])
def test_mixed_projection_order3_tile_edges(cuda_lib, kind):
    """Order-3 projection at the edges of the fused kernel's tiling: b_1 = 21 (not a multiple of
    its 4-row blocks), core slices split into several mode-3 chunks (r_1 r_2 = 1920 > 1024),
    rank-1 terms, and a problem whose b_3 > 64 takes the tensor-core path for the last mode."""
    g = np.random.default_rng(77)
    specs = [([56, 48, 40], [[48, 40, 37], [1, 1, 1], [5, 33, 17]], [10, 15, 8], [3, 6, 3]),
             ([72, 64, 80], [[8, 8, 8], [20, 3, 30]], [60, 56, 62], [6, 6, 6])]
    probs = []
    for dims, ranks, target, over in specs:
        cores = [g.standard_normal(r) for r in ranks]
        facs = [[g.standard_normal((n, ri)) for n, ri in zip(dims, r)] for r in ranks]
        probs.append(wl.Problem(dims, cores, facs, target, over, alpha=list(g.standard_normal(len(ranks)))))
    probs = wl._finish(probs, True)
    plan = _plan(probs, kind, 8)
    refs = [_oracle(p, kind, 8, i) for i, p in enumerate(probs)]
    Hs = plan.project([r["Q"] for r in refs])
    for H, r in zip(Hs, refs):
        assert H.shape == r["H"].shape
        assert _rel(H, r["H"]) <= 1e-5, _rel(H, r["H"])
        _per_slice(H, r["H"], 1e-5)


@pytest.mark.parametrize("precision", MODES)
@pytest.mark.parametrize("d", [3, 4])
def test_mixed_projection_of_an_arbitrary_given_basis(cuda_lib, precision, d):
    """tks_project_core with caller-given orthonormal bases that no QR of this plan produced,
    called on a fresh plan before any recompression: the bf16 planes of Q must come from the given
    Q (the register QR writes them only inside the recompression)."""
    probs = _bf16_problems(d, 3)
    plan = _plan(probs, "krp", 13, precision=precision)
    g = np.random.default_rng(14)
    Qs = [[wl.haar(g, n, b) for n, b in zip(p.dims, pi.basis_cols)] for p, pi in zip(probs, plan.pinfo)]
    Hs = plan.project(Qs)
    for p, Q, H in zip(probs, Qs, Hs):
        ref = ss.project_core(ss.scaled_terms(p.terms(), p.alpha), Q)
        assert _rel(H, ref) <= 1e-5, _rel(H, ref)


@pytest.mark.parametrize("precision", MODES)
@pytest.mark.parametrize("kind", ["kron", "krp"])
def test_mixed_recompress_small(cuda_lib, kind, precision):
    probs = _bf16_problems(3, 2)
    outs = _plan(probs, kind, 7, precision=precision).recompress()
    for i, (prob, got) in enumerate(zip(probs, outs)):
        ref = _oracle(prob, kind, 7, i)
        X = sum(a * tucker_full(G, Us) for a, (G, Us) in zip(prob.alpha, prob.terms()))
        Xg = tucker_full(got["core"], got["factors"])
        Xo = tucker_full(ref["core"], ref["factors"])
        nx = np.linalg.norm(X)
        assert np.linalg.norm(Xg - Xo) / nx <= 1e-5
        assert abs(np.linalg.norm(Xg - X) - np.linalg.norm(Xo - X)) / nx <= 1e-5
        assert got["ranks"] == ref["ranks"]


@pytest.mark.parametrize("precision", MODES)
def test_mixed_recompress_short_modes(cuda_lib, precision):
    """Modes with fewer rows than sketch columns (n_1 = 16 < S = 20, so b_1 = n_1 and the QR of Y_1
    is wide) next to rows-per-lane boundaries of the float32 QR kernels (n = 128, 136, 256, 264)."""
    g = np.random.default_rng(79)
    specs = [([16, 24, 64], 5, [12, 12, 12], [8, 8, 8]), ([128, 136, 256], 4, [10, 10, 10], [4, 4, 4]),
             ([264, 40, 32], 3, [8, 8, 8], [3, 3, 3])]
    probs = []
    for dims, K, target, over in specs:
        ranks = [[int(min(x, n)) for x, n in zip(g.integers(2, 9, size=3), dims)] for _ in range(K)]
        cores = [g.standard_normal(r) for r in ranks]
        facs = [[g.standard_normal((n, ri)) for n, ri in zip(dims, r)] for r in ranks]
        probs.append(wl.Problem(dims, cores, facs, target, over, alpha=list(g.standard_normal(K))))
    probs = wl._finish(probs, True)
    outs = _plan(probs, "krp", 12, precision=precision).recompress()
    for i, (prob, got) in enumerate(zip(probs, outs)):
        ref = _oracle(prob, "krp", 12, i)
        assert got["ranks"] == ref["ranks"]
        X = sum(a * tucker_full(G, Us) for a, (G, Us) in zip(prob.alpha, prob.terms()))
        Xg = tucker_full(got["core"], got["factors"])
        Xo = tucker_full(ref["core"], ref["factors"])
        nx = np.linalg.norm(X)
        assert np.linalg.norm(Xg - Xo) / nx <= 1e-5, (i, np.linalg.norm(Xg - Xo) / nx)


@pytest.mark.parametrize("precision", MODES)
def test_mixed_decay512_full_size(cuda_lib, precision):
    w = wl.decay512()
    p = w.problems[0]
    plan = _plan(w.problems, "krp", w.seed, precision=precision)
    ref = _oracle(p, "krp", w.seed, 0)
    Ys = plan.sketch()[0]
    for m in range(3):
        assert _rel(Ys[m], ref["Y"][m]) <= 1e-5
    assert _rel(plan.project([ref["Q"]])[0], ref["H"]) <= 1e-5
    got = plan.recompress()[0]
    assert got["ranks"] == ref["ranks"] == [48, 48, 48]
    idx = np.random.default_rng(1).integers(0, 512, size=(400, 3))
    eg = tucker_entries(got["core"], got["factors"], idx)
    eo = tucker_entries(ref["core"], ref["factors"], idx)
    ex = sum(tucker_entries(G, Us, idx) for G, Us in p.terms())
    scale = np.sqrt(np.mean(ex ** 2))
    assert np.sqrt(np.mean((eg - eo) ** 2)) <= 1e-5 * scale
    # both truncations are ~1e-6 of ||X|| here; their sampled errors agree to 1e-5
    assert abs(np.sqrt(np.mean((eg - ex) ** 2)) - np.sqrt(np.mean((eo - ex) ** 2))) <= 1e-5 * scale


@pytest.mark.parametrize("precision", MODES)
def test_mixed_tolerance_rule_and_d4(cuda_lib, precision):
    # Sec. 5.1.1-style low rank that survives bf16 rounding: every term uses the same bf16 basis
    # Q_m (n x 10) and a rank-1 bf16 core, so each mode of the sum has rank 10 exactly
    g = np.random.default_rng(4)
    dims = [64, 48, 56, 40]
    Qs = [wl.to_bf16_values(wl.haar(g, n, 10)) for n in dims]
    cores = []
    for _ in range(20):
        vs = [g.standard_normal(10) for _ in dims]
        cores.append(wl.to_bf16_values(np.einsum("a,b,c,d->abcd", *vs)))
    prob = wl.Problem(dims, cores, [list(Qs) for _ in cores], [10] * 4, [2] * 4)
    got = _plan([prob], "krp", 11, tol=1e-6, precision=precision).recompress()[0]
    assert got["ranks"] == [10, 10, 10, 10]
    X = tucker_sum_full(prob.terms())
    assert np.linalg.norm(tucker_full(got["core"], got["factors"]) - X) <= 1e-5 * np.linalg.norm(X)


def test_mixed_rejects_unaligned_mode_size(cuda_lib):
    from paper_2603_13532_gb300 import binding
    g = np.random.default_rng(3)
    dims = [20, 16, 16]
    p = wl.Problem(dims, [g.standard_normal((2, 2, 2))], [[g.standard_normal((n, 2)) for n in dims]],
                   [3, 3, 3], [1, 1, 1])
    with pytest.raises(binding.TksError) as e:
        _plan(wl._finish([p], True), "krp", 1)
    assert e.value.code == 7


@pytest.mark.parametrize("precision", ["fp64"] + MODES)
@pytest.mark.parametrize("kind", ["krp", "kron"])
@pytest.mark.parametrize("d", [5, 6])
def test_high_order_recompress_matches_oracle(cuda_lib, precision, kind, d):
    """Orders 5 and 6 (the generic chain path of every precision) against the oracle on the same
    draws: entrywise for float64, and reconstruction plus truncation error for the mixed modes."""
    g = np.random.default_rng(400 + d)
    dims = [8, 16, 8, 16, 8, 8][:d]
    cores, facs = [], []
    for _ in range(3):
        r = [int(x) for x in g.integers(1, 4, size=d)]
        cores.append(g.standard_normal(r))
        facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
    prob = wl.Problem(dims, cores, facs, [3] * d, [2] * d, alpha=list(g.standard_normal(3)))
    bf16 = precision != "fp64"
    prob = wl._finish([prob], bf16)[0]
    got = _plan([prob], kind, 21, precision=precision).recompress()[0]
    ref = ss.recompress(prob.terms(), kind, prob.target, prob.oversampling, seed=21, alpha=prob.alpha,
                        rounding="bf16" if bf16 else None)
    assert got["ranks"] == ref["ranks"]
    X = sum(a * tucker_full(G, Us) for a, (G, Us) in zip(prob.alpha, prob.terms()))
    Xg = tucker_full(got["core"], got["factors"])
    Xo = tucker_full(ref["core"], ref["factors"])
    nx = np.linalg.norm(X)
    tol = 1e-11 if precision == "fp64" else 1e-5
    assert np.linalg.norm(Xg - Xo) / nx <= tol, np.linalg.norm(Xg - Xo) / nx
    assert abs(np.linalg.norm(Xg - X) - np.linalg.norm(Xo - X)) / nx <= tol


@pytest.mark.parametrize("precision", MODES)
def test_lanes_give_identical_results(cuda_lib, precision):
    # the same problems split into 3 lanes on concurrent streams (eager and CUDA-graph replay) give
    # bit-identical outputs to one launch sequence: every problem's arithmetic is per problem
    import torch
    from paper_2603_13532_gb300 import binding
    probs = _bf16_problems(3) + _bf16_problems(3, seed=1) + wl.decay512(num_problems=2).problems
    one = binding.Plan(probs, kind="krp", precision=precision, seed=5)
    ref = one.recompress()
    three = binding.Plan(probs, kind="krp", precision=precision, seed=5, lanes=3)
    assert three.info.launches_recompress > one.info.launches_recompress
    got = three.recompress()
    for a, b in zip(got, ref):
        assert a["ranks"] == b["ranks"]
        assert np.array_equal(a["core"], b["core"])
        for fa, fb in zip(a["factors"], b["factors"]):
            assert np.array_equal(fa, fb)
    out = torch.zeros(three.info.output_elems, dtype=torch.float64, device="cuda")
    ranks = torch.zeros(len(probs) * binding.MAX_ORDER, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        three.recompress_raw(out, ranks)
    torch.cuda.current_stream().wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        three.recompress_raw(out, ranks)
    out.zero_()
    graph.replay()
    torch.cuda.synchronize()
    three.sync()
    for a, b in zip(three.unpack(out, ranks), ref):
        assert a["ranks"] == b["ranks"] and np.array_equal(a["core"], b["core"])


@pytest.mark.parametrize("precision", ["fp64"] + MODES)
@pytest.mark.parametrize("kind,ell", [("krp", 96), ("kron", 81)])
def test_limits_rank64_basis96(cuda_lib, precision, kind, ell):
    # a term of rank 64 (TKS_MAX_RANK) and sketches with up to 96 columns (TKS_MAX_BASIS for the
    # Khatri-Rao case; the Kronecker sizes of ell = 81 give S_n = 81): every stage runs its
    # general kernels (no rank-32 / basis-64 fast paths).  The sum has multilinear rank 74, below
    # both targets (90 and 75), so the recompression reproduces it; checked against the dense sum
    # and the oracle.
    from paper_2603_13532_gb300 import binding
    g = np.random.default_rng(64)
    n = 128
    ranks = [(64, 64, 64), (8, 8, 8), (2, 2, 2)]
    cores = [g.standard_normal(r) for r in ranks]
    facs = [[wl.haar(g, n, ri) for ri in r] for r in ranks]
    target = ell - 6
    p = wl.Problem([n] * 3, cores, facs, [target] * 3, [6] * 3)
    if precision != "fp64":
        p = wl._finish([p], True)[0]
    plan = binding.Plan([p], kind=kind, precision=precision, seed=3)
    assert [plan.pinfo[0].basis_cols[m] for m in range(3)] == [96 if kind == "krp" else 81] * 3
    got = plan.recompress()[0]
    ref = ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=3,
                        rounding=None if precision == "fp64" else "bf16")
    X = tucker_sum_full(p.terms())
    nx = np.linalg.norm(X)
    Xg = tucker_full(got["core"], got["factors"])
    Xo = tucker_full(ref["core"], ref["factors"])
    tol = 1e-11 if precision == "fp64" else 1e-5
    assert np.linalg.norm(Xg - X) <= tol * nx
    assert np.linalg.norm(Xg - Xo) <= tol * nx
    assert got["ranks"] == ref["ranks"] == [target] * 3

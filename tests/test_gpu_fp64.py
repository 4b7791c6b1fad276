"""GPU parity of the plain FP64 path (TKS_FP64) against the FP64 CPU oracle, through the C ABI.

Tolerances
  Omega                bit-exact (same IEEE operations in the same order on both sides)
  Y_n, H (given Q)     1e-12 relative Frobenius: both are sums of products of O(1) numbers
                       evaluated in float64 in different orders
  Q_n                  projector difference 1e-12 on well-conditioned sketches (Q is unique
                       only up to the sign convention diag(R) >= 0 both sides use)
  recompression        1e-12 relative (reconstructions, or sampled entries of them, against the
                       oracle's): both sides take the ST-HOSVD from a backward-stable SVD of each
                       unfolding (TSQR + one-sided Jacobi here, LAPACK there), so the kept subspaces
                       differ by eps ||H|| / gap in angle and the reconstructions by about
                       eps ||H|| sigma_r / gap, a few eps of ||X|| at the decay512 truncation point
"""
import json
import os

import numpy as np
import pytest

from oracle import rng
from oracle import sketch_sum as ss
from oracle.tensor import tucker_entries, tucker_full, tucker_sum_full
from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _plan(w, problems=None, **kw):
    from paper_2603_13532_gb300 import binding
    args = dict(kind=w.kind, precision="fp64", seed=w.seed, tol=w.tol)
    args.update(kw)
    return binding.Plan(problems if problems is not None else w.problems, **args)


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


def _ragged_problems(d, kind_seed=0):
    g = np.random.default_rng(100 + d + kind_seed)
    probs = []
    for dims, K in ([[70, 33, 129, 41][:d], 3], [[17, 65, 9, 23][:d], 2], [[100] * d, 5]):
        cores, facs = [], []
        for _ in range(K):
            r = [int(x) for x in g.integers(1, 8, size=d)]
            r = [min(ri, n) for ri, n in zip(r, dims)]
            cores.append(g.standard_normal(r))
            facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
        probs.append(wl.Problem(list(dims), cores, facs, [6] * d, [2] * d,
                                alpha=list(g.standard_normal(K))))
    return probs


def test_omega_bit_exact(cuda_lib):
    w = wl.exact_recovery(n=37, K=2, r=3, target=9)
    probs = _ragged_problems(3) + w.problems
    for kind in ("krp", "kron"):
        plan = _plan(w, probs, kind=kind, seed=20260315)
        om = plan.omega()
        for p, (prob, pi) in enumerate(zip(probs, plan.pinfo)):
            for m in range(prob.order):
                ref = rng.omega(20260315, p, m, prob.dims[m], pi.omega_cols[m])
                assert om[p][m].shape == ref.shape
                assert np.array_equal(om[p][m].view(np.uint64), ref.view(np.uint64)), (kind, p, m)


def test_omega_matches_golden_heads(cuda_lib):
    gold = json.load(open(os.path.join(HERE, "golden", "omega_head.json")))
    for entry in gold["draws"]:
        p = entry["problem"]
        # a plan whose problem p has mode entry["mode"] with n * s >= 32 draws
        probs = [wl.exact_recovery(n=16, K=1, r=2, target=2).problems[0] for _ in range(p + 1)]
        for q in probs:
            q.target = [4, 4, 4]
            q.oversampling = [0, 0, 0]
        plan = _plan(wl.exact_recovery(), probs, kind="krp", seed=entry["seed"])
        om = plan.omega()[p][entry["mode"]].ravel(order="F")[:32]
        want = np.array([float.fromhex(h) for h in entry["values"]])
        assert np.array_equal(om, want)


@pytest.mark.parametrize("kind", ["krp", "kron"])
@pytest.mark.parametrize("d", [2, 3, 4])
def test_sketch_matches_oracle(cuda_lib, kind, d):
    probs = _ragged_problems(d)
    plan = _plan(wl.exact_recovery(), probs, kind=kind, seed=7)
    Ys = plan.sketch()
    for p, prob in enumerate(probs):
        ref = ss.recompress(prob.terms(), kind, prob.target, prob.oversampling, seed=7, problem=p,
                            alpha=prob.alpha)
        for m in range(d):
            assert _rel(Ys[p][m], ref["Y"][m]) <= 1e-12, (kind, d, p, m)
            _per_slice(Ys[p][m], ref["Y"][m], 1e-12)


@pytest.mark.parametrize("kind", ["krp", "kron"])
@pytest.mark.parametrize("d", [2, 3, 4])
def test_projection_matches_oracle_given_q(cuda_lib, kind, d):
    probs = _ragged_problems(d, 1)
    plan = _plan(wl.exact_recovery(), probs, kind=kind, seed=8)
    refs = [ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=8, problem=i, alpha=p.alpha)
            for i, p in enumerate(probs)]
    Hs = plan.project([r["Q"] for r in refs])
    for H, r in zip(Hs, refs):
        assert H.shape == r["H"].shape
        assert _rel(H, r["H"]) <= 1e-12
        _per_slice(H, r["H"], 1e-12)


@pytest.mark.parametrize("kind", ["kron", "krp"])
def test_recompress_exact_recovery(cuda_lib, kind):
    w = wl.exact_recovery()
    p = w.problems[0]
    got = _plan(w, kind=kind).recompress()[0]
    ref = ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=w.seed)
    X = tucker_sum_full(p.terms())
    Xg = tucker_full(got["core"], got["factors"])
    assert _rel(Xg, X) <= 1e-12
    assert _rel(Xg, tucker_full(ref["core"], ref["factors"])) <= 1e-12
    assert got["ranks"] == ref["ranks"]


def test_recompress_batched_ragged_problems(cuda_lib):
    probs = _ragged_problems(3, 2) + _ragged_problems(4, 3)[:2]
    plan = _plan(wl.exact_recovery(), probs, kind="krp", seed=9)
    outs = plan.recompress()
    for i, (prob, got) in enumerate(zip(probs, outs)):
        ref = ss.recompress(prob.terms(), "krp", prob.target, prob.oversampling, seed=9, problem=i,
                            alpha=prob.alpha)
        assert got["ranks"] == ref["ranks"]
        X = sum(a * tucker_full(G, Us) for a, (G, Us) in zip(prob.alpha, prob.terms()))
        Xo = tucker_full(ref["core"], ref["factors"])
        Xg = tucker_full(got["core"], got["factors"])
        # target 6 is below the sum's ranks here: compare against the oracle's truncation
        assert _rel(Xg, Xo) <= 1e-12 * max(1.0, np.linalg.norm(X) / np.linalg.norm(Xo))


def test_recompress_tolerance_rule(cuda_lib):
    w = wl.shared_subspace(n=60, K=20, d=4)
    p = w.problems[0]
    got = _plan(w).recompress()[0]
    assert got["ranks"] == [10, 10, 10, 10]
    X = tucker_sum_full(p.terms())
    assert _rel(tucker_full(got["core"], got["factors"]), X) <= 1e-12


def test_edge_cases_rank_one_single_term_wide_sketch(cuda_lib):
    g = np.random.default_rng(5)
    dims = [6, 9, 5]
    # K = 1, rank-1 term; KRP sketch s = 12 wider than n_1 and n_3 (b_n = min(n_n, s))
    one = wl.Problem(dims, [np.array([[[2.5]]])], [[g.standard_normal((n, 1)) for n in dims]],
                     [10, 10, 10], [2, 2, 2])
    plan = _plan(wl.exact_recovery(), [one], kind="krp", seed=3)
    got = plan.recompress()[0]
    X = tucker_sum_full(one.terms())
    assert got["ranks"] == [6, 9, 5]        # target mode keeps rmax_n = min(target_n, b_n)
    assert _rel(tucker_full(got["core"], got["factors"]), X) <= 1e-12
    assert [pi for pi in plan.pinfo[0].basis_cols][:3] == [6, 9, 5]


def test_decay512_fp64_full_size(cuda_lib):
    w = wl.decay512(bf16=False)
    p = w.problems[0]
    plan = _plan(w)
    ref = ss.recompress(p.terms(), w.kind, p.target, p.oversampling, seed=w.seed)
    Ys = plan.sketch()[0]
    for m in range(3):
        assert _rel(Ys[m], ref["Y"][m]) <= 1e-12
    H = plan.project([ref["Q"]])[0]
    assert _rel(H, ref["H"]) <= 1e-12
    got = plan.recompress()[0]
    assert got["ranks"] == ref["ranks"] == [48, 48, 48]
    # sampled entries of the reconstructions (the dense 512^3 tensor is not formed)
    idx = np.random.default_rng(0).integers(0, 512, size=(400, 3))
    eg = tucker_entries(got["core"], got["factors"], idx)
    eo = tucker_entries(ref["core"], ref["factors"], idx)
    ex = sum(tucker_entries(G, Us, idx) for G, Us in p.terms())
    scale = np.sqrt(np.mean(ex ** 2))
    assert np.max(np.abs(eg - eo)) <= 1e-12 * scale

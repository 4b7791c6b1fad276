"""GPU parity of the effective subrank heuristic (Alg. 5) through the C ABI.

The ranks are integers decided in float64 on both sides (oracle: LAPACK's symmetric solver on
the R_n x R_n Gram matrix; library: the smaller of V^T V and V V^T, Householder tridiagonal
reduction and implicit QR steps).  Both are backward stable, so every eigenvalue agrees to a
few units of u ||B|| (the test allows 1e-12 lambda_max); the ranks must be identical wherever
the threshold tau is not within that distance of a tail sum, which the tests ensure by
choosing eps in the middle of a gap of the oracle's tail sums.

  closed form   block-orthogonal factors, ranks for eps values worked out by hand
  shapes        Gram orders across the 64-wide tiles and the tridiagonal kernel's 1/2/4 rows
                per thread (m up to 1100), both Gram forms (R <= n and n < R), orders 2 and 4
  bf16          decay512 problems with bfloat16 inputs, eps from the oracle's gaps and the
                paper's eps = 1e-6
  edges         a single rank-1 term (m = 1), all-zero cores, huge eps, negative alpha
  end to end    Alg. 4 as printed: ell from the heuristic, then the plan with tol = eps
"""
import numpy as np
import pytest

from oracle import sketch_sum as ss
from oracle import subrank as sr
from oracle.tensor import tucker_entries
from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _gpu(problems, eps, dtype="fp64", eigenvalues=True):
    from paper_2603_13532_gb300 import binding
    return binding.SubrankPlan(problems, eps, dtype=dtype).run(eigenvalues=eigenvalues)


def _problem(terms, over, alpha=None):
    d = len(terms[0][1])
    return wl.Problem([terms[0][1][m].shape[0] for m in range(d)], [G for G, _ in terms], [Us for _, Us in terms],
                      [1] * d, list(over), alpha)


def _random_terms(seed, dims, K, rmin, rmax, decay=0.0):
    g = np.random.default_rng(seed)
    terms = []
    for k in range(K):
        r = [int(x) for x in g.integers(rmin, rmax + 1, size=len(dims))]
        G = g.standard_normal(r) * 10.0 ** (-decay * k)
        terms.append((G, [g.standard_normal((n, rm)) / np.sqrt(n) for n, rm in zip(dims, r)]))
    return terms


def _check_eigenvalues(got_lam, ref_lam):
    # the library's m = min(n, R) eigenvalues against the top m of the oracle's R (the rest are 0)
    m = len(got_lam)
    ref = np.asarray(ref_lam)
    assert np.all(ref[m:] <= 1e-12 * ref[0] + 1e-300)
    np.testing.assert_allclose(np.maximum(got_lam, 0.0), ref[:m], rtol=0, atol=1e-12 * ref[0])


def _gap_eps(lam, rank, order):
    """eps whose threshold sits halfway (geometrically) between tail(rank) and tail(rank - 1)."""
    lam = np.asarray(lam)
    total = float(np.sum(lam))
    lo, hi = float(np.sum(lam[rank:])), float(np.sum(lam[rank - 1:]))
    tau = np.sqrt(max(lo, 1e-300) * hi)
    return float(np.sqrt(tau * order / total))


# ------------------------------------------------------------------ closed form
def _block_terms(seed, n, ranks_per_term, weights):
    rng = np.random.default_rng(seed)
    d = len(ranks_per_term[0])
    totals = [sum(r[m] for r in ranks_per_term) for m in range(d)]
    bases = [wl.haar(rng, n, totals[m]) for m in range(d)]
    offs = [0] * d
    terms = []
    for r, w in zip(ranks_per_term, weights):
        Z = rng.standard_normal(tuple(r))
        G = Z * (w / np.sqrt(np.sum(Z * Z)))
        Us = []
        for m in range(d):
            Us.append(bases[m][:, offs[m]:offs[m] + r[m]])
            offs[m] += r[m]
        terms.append((G, Us))
    return terms


@pytest.mark.parametrize("eps,rank0", [(2.0, 1), (0.35, 5), (0.3, 6), (1e-3, 7), (1e-6, 12)])
def test_closed_form(cuda_lib, eps, rank0):
    ranks = [(3, 4, 1), (2, 1, 5), (2, 2, 2), (5, 3, 1)]
    terms = _block_terms(1, 40, ranks, [4.0, 2.0, 1.0, 1e-4])
    got = _gpu([_problem(terms, [3, 3, 3])], eps)[0]
    assert got["rank"][0] == rank0
    assert got["ell"][0] == rank0 + 3
    np.testing.assert_allclose(got["lam"][0], [16.0] * 3 + [4.0] * 2 + [1.0] * 2 + [1e-8] * 5, rtol=1e-12, atol=1e-14)
    ref = sr.effective_subrank(terms, eps, [3, 3, 3])
    assert got["rank"] == ref["rank"] and got["ell"] == ref["ell"]


# ------------------------------------------------------------------ shapes
SHAPES = [
    # (dims, K, rmin, rmax): Gram orders m_n = min(n_n, R_n)
    ((40, 30, 20), 3, 1, 4),          # tiny, R <= n
    ((64, 64, 64), 8, 8, 8),          # m = 64 = one tile
    ((60, 70, 300), 13, 5, 5),        # m = 60 (n < R: V V^T), then R = 65 <= n twice
    ((130, 96, 300), 12, 10, 12),     # ragged tiles, both forms
    ((600, 520, 600), 40, 12, 16),    # m > 512: two rows per thread
    ((1100, 1100), 70, 16, 16),       # order 2, m = 1100 > 1024: four rows per thread
    ((50, 40, 30, 20), 6, 2, 6),      # order 4
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s[0])) + f"_K{s[1]}")
def test_shapes_against_oracle(cuda_lib, shape):
    dims, K, rmin, rmax = shape
    terms = _random_terms(hash(dims) % 1000, dims, K, rmin, rmax, decay=0.15)
    d = len(dims)
    over = [2] * d
    ref = sr.effective_subrank(terms, 1e-3, over)
    prob = _problem(terms, over)
    got = _gpu([prob], 1e-3)[0]
    for m in range(d):
        _check_eigenvalues(got["lam"][m], ref["lam"][m])
    # eps placed in gaps of mode 0's tail sums at a few ranks
    m_eff = min(dims[0], sum(U[0].shape[1] for _, U in terms))
    for target in sorted({1, 2, max(1, m_eff // 3), max(1, m_eff // 2)}):
        eps = _gap_eps(ref["lam"][0], target, d)
        r_ref = sr.effective_subrank(terms, eps, over)
        assert r_ref["rank"][0] == target
        r_got = _gpu([prob], eps, eigenvalues=False)[0]
        assert r_got["rank"] == r_ref["rank"], (eps, r_got, r_ref["rank"])
        assert r_got["ell"] == r_ref["ell"]


def test_many_problems_in_one_plan(cuda_lib):
    probs, refs = [], []
    for i, (dims, K, rmin, rmax) in enumerate(SHAPES[:5]):
        terms = _random_terms(100 + i, dims, K, rmin, rmax, decay=0.2)
        over = [i % 3] * len(dims)
        probs.append(_problem(terms, over, alpha=list(np.linspace(-2.0, 3.0, K))))
        refs.append(sr.effective_subrank(terms, 1e-4, over, alpha=probs[-1].alpha))
    got = _gpu(probs, 1e-4)
    for g, r in zip(got, refs):
        for m in range(len(r["lam"])):
            _check_eigenvalues(g["lam"][m], r["lam"][m])
        # the rank is only compared where tau is not at a tail sum to within the eigenvalue error
        for m in range(len(r["lam"])):
            lam = np.asarray(r["lam"][m])
            k = r["rank"][m]
            tail_in, tail_out = float(np.sum(lam[k:])), float(np.sum(lam[k - 1:]))
            tau = r["tau"][m]
            if tail_out - tau > 1e-9 * lam[0] and tau - tail_in > 1e-9 * lam[0]:
                assert g["rank"][m] == k
                assert g["ell"][m] == r["ell"][m]


# ------------------------------------------------------------------ bf16 inputs (decay512)
def test_decay512_bf16(cuda_lib):
    w = wl.decay512(num_problems=3)
    from paper_2603_13532_gb300 import binding
    plan = binding.SubrankPlan(w.problems, 1e-6, dtype="bf16")
    got = plan.run(eigenvalues=True)
    for p, g in zip(w.problems, got):
        ref = sr.effective_subrank(p.terms(), 1e-6, p.oversampling)
        for m in range(3):
            assert len(g["lam"][m]) == 512   # R ~ 640 > n: the n x n form
            _check_eigenvalues(g["lam"][m], ref["lam"][m])
            lam = np.asarray(ref["lam"][m])
            k = ref["rank"][m]
            if float(np.sum(lam[k - 1:])) - ref["tau"][m] > 1e-9 * lam[0] and \
                    ref["tau"][m] - float(np.sum(lam[k:])) > 1e-9 * lam[0]:
                assert g["rank"][m] == k
        for target in (10, 30):
            eps = _gap_eps(ref["lam"][0], target, 3)
            r_ref = sr.effective_subrank(p.terms(), eps, p.oversampling)
            r_got = binding.SubrankPlan([p], eps, dtype="bf16").run()[0]
            assert r_got["rank"][0] == r_ref["rank"][0] == target


def test_executed_flops_count_the_early_end(cuda_lib):
    """decay512's Gram matrices (n = 512, rank ~128) end their reduction early: the executed count lies
    between the Gram flops alone and the algorithmic count (stopping after ~130 of 511 steps still runs
    the costliest steps, about 60% of a full reduction's flops); a full-rank matrix runs every step, so
    its executed count is the full reduction (sum_k 4 (m - k)^2, k < m - 1)."""
    from paper_2603_13532_gb300 import binding
    w = wl.decay512(num_problems=2)
    plan = binding.SubrankPlan(w.problems, 1e-6, dtype="bf16")
    plan.run()
    ex = plan.executed_flops()
    full = 6 * 4.0 / 3.0 * 512.0 ** 3
    gram = plan.info.flops - full   # the algorithmic count less the full reductions
    assert gram < ex < gram + 0.8 * full
    g = np.random.default_rng(6)
    dims, r = [40, 40, 40], 12
    p = wl.Problem(dims, [g.standard_normal((r, r, r)) for _ in range(5)],
                   [[g.standard_normal((n, r)) for n in dims] for _ in range(5)], [4, 4, 4], [2, 2, 2])
    whole = binding.SubrankPlan([p], 1e-6, dtype="fp64")
    whole.run()
    m = 40   # R = 60 > n = 40: the n x n form, full rank
    red = sum(4.0 * (m - k) ** 2 for k in range(m - 1))
    gram_f = 3 * 2.0 * 60 * 0.5 * m * (m + 1)
    assert abs(whole.executed_flops() - (gram_f + 3 * red)) <= 1e-9 * whole.executed_flops()


# ------------------------------------------------------------------ edges
def test_edges(cuda_lib):
    g = np.random.default_rng(5)
    # one rank-1 term: every Gram matrix is 1 x 1
    t1 = [(np.array([[[2.5]]]), [g.standard_normal((7, 1)) for _ in range(3)])]
    got = _gpu([_problem(t1, [4, 0, 1])], 1e-6)[0]
    assert got["rank"] == [1, 1, 1] and got["ell"] == [5, 1, 2]
    for m in range(3):
        np.testing.assert_allclose(got["lam"][m], [6.25 * float(t1[0][1][m][:, 0] @ t1[0][1][m][:, 0])], rtol=1e-13)
    # all-zero cores: every eigenvalue is zero, tau = 0, rank 1
    t0 = [(np.zeros((3, 2, 2)), [g.standard_normal((9, r)) for r in (3, 2, 2)]) for _ in range(2)]
    got = _gpu([_problem(t0, [1, 1, 1])], 1e-6)[0]
    assert got["rank"] == [1, 1, 1]
    # huge eps: rank 1 everywhere; alpha signs do not matter
    terms = _random_terms(9, (30, 31, 32), 5, 2, 6)
    got = _gpu([_problem(terms, [0, 0, 0])], 50.0)[0]
    assert got["rank"] == [1, 1, 1]
    # cores scaled by 1e-100 and 1e+100: Gram entries near 1e-200 and 1e+200 (the Householder norms
    # and the tridiagonal QR are scaled internally); same ranks, eigenvalues scaled by 1e-+200
    base = _gpu([_problem(terms, [0, 0, 0])], 1e-5)[0]
    for f in (1e-100, 1e100):
        got_s = _gpu([_problem([(f * G, Us) for G, Us in terms], [0, 0, 0])], 1e-5)[0]
        ref_s = sr.effective_subrank([(f * G, Us) for G, Us in terms], 1e-5, [0, 0, 0])
        assert got_s["rank"] == base["rank"] == ref_s["rank"]
        for m in range(3):
            _check_eigenvalues(got_s["lam"][m], ref_s["lam"][m])
    a = [1.0, -2.0, 0.5, -0.25, 3.0]
    got_p = _gpu([_problem(terms, [0, 0, 0], alpha=[abs(x) for x in a])], 1e-5)[0]
    got_n = _gpu([_problem(terms, [0, 0, 0], alpha=a)], 1e-5)[0]
    assert got_p["rank"] == got_n["rank"]
    for m in range(3):
        np.testing.assert_allclose(got_n["lam"][m], got_p["lam"][m], rtol=0, atol=1e-13 * got_p["lam"][m][0])


# ------------------------------------------------------------------ Alg. 4 as printed
def test_krpsum_with_effective_ranks(cuda_lib):
    from paper_2603_13532_gb300 import binding
    w = wl.shared_subspace(K=12, n=120, d=3)
    p = w.problems[0]
    eps = 1e-6
    sub = binding.SubrankPlan([p], eps).run()[0]
    ref_sub = sr.effective_subrank(p.terms(), eps, p.oversampling)
    assert sub["ell"] == ref_sub["ell"]
    q = binding.with_sketch_ranks([p], [sub["ell"]])[0]
    got = binding.Plan([q], kind="krp", precision="fp64", seed=w.seed, tol=eps).recompress()[0]
    ref = ss.recompress(p.terms(), "krp", q.target, q.oversampling, seed=w.seed, tol=eps)
    assert got["ranks"] == ref["ranks"] == [10, 10, 10]
    idx = np.stack([np.random.default_rng(0).integers(0, n, size=200) for n in p.dims], axis=1)
    ex = sum(tucker_entries(G, Us, idx) for G, Us in p.terms())
    eg = tucker_entries(got["core"], got["factors"], idx)
    assert np.sqrt(np.mean((eg - ex) ** 2)) <= 1e-10 * np.sqrt(np.mean(ex ** 2))


# ------------------------------------------------------------------ full-size batches, sampled
def _sampled_parity(problems, got, eps, picks):
    for i in picks:
        p, g = problems[i], got[i]
        ref = sr.effective_subrank(p.terms(), eps, p.oversampling, alpha=p.alpha)
        for m in range(p.order):
            _check_eigenvalues(g["lam"][m], ref["lam"][m])
            lam = np.asarray(ref["lam"][m])
            k = ref["rank"][m]
            tau = ref["tau"][m]
            # the rank where tau is not within the eigenvalue error of a tail sum
            if float(np.sum(lam[k - 1:])) - tau > 1e-9 * lam[0] and tau - float(np.sum(lam[k:])) > 1e-9 * lam[0]:
                assert g["rank"][m] == k, (i, m, g["rank"], ref["rank"])
                assert g["ell"][m] == ref["ell"][m]


def test_decay512_152_problems(cuda_lib):
    # the bench's launch: 152 decay512 problems (one plan, bf16 inputs, eps = 1e-6), 4 checked
    from paper_2603_13532_gb300 import binding
    import bench
    probs = bench.make_problems(152, 20260315, 0, True, "decay512")
    got = binding.SubrankPlan(probs, 1e-6, dtype="bf16").run(eigenvalues=True)
    assert all(1 <= r <= 512 for g in got for r in g["rank"])
    _sampled_parity(probs, got, 1e-6, [0, 51, 102, 151])


def test_batched_256_problems(cuda_lib):
    # the batched workload at full size: 256 problems, n up to 1024, K up to 48 (Gram orders up to
    # 1024, both Gram forms), 4 problems checked, the largest among them
    from paper_2603_13532_gb300 import binding
    w = wl.batched()
    got = binding.SubrankPlan(w.problems, 1e-5, dtype="bf16").run(eigenvalues=True)
    orders = [min(p.dims[0], sum(r[0] for r in p.ranks())) for p in w.problems]
    big = int(np.argmax(orders))
    _sampled_parity(w.problems, got, 1e-5, sorted({0, 100, 200, big}))


def test_kronsum_with_effective_ranks(cuda_lib):
    # Alg. 3 as printed on the exact-recovery workload (K = 4 terms of rank 8, Kronecker sketch):
    # the heuristic finds rank 32 = sum of the term ranks in every mode, the Kronecker sizes follow
    # from ell, and the recompression recovers the sum
    from paper_2603_13532_gb300 import binding
    from oracle.tensor import tucker_full, tucker_sum_full
    w = wl.exact_recovery()
    p = w.problems[0]
    eps = 1e-8
    sub = binding.SubrankPlan([p], eps).run()[0]
    ref_sub = sr.effective_subrank(p.terms(), eps, p.oversampling, kind="kron")
    assert sub["rank"] == ref_sub["rank"] == [32, 32, 32]
    q = binding.with_sketch_ranks([p], [sub["ell"]])[0]
    plan = binding.Plan([q], kind="kron", precision="fp64", seed=w.seed, tol=eps)
    assert [plan.pinfo[0].omega_cols[m] for m in range(3)] == ref_sub["cols"]
    got = plan.recompress()[0]
    X = tucker_sum_full(p.terms())
    err = np.linalg.norm(tucker_full(got["core"], got["factors"]) - X) / np.linalg.norm(X)
    assert err <= 1e-12 and got["ranks"] == [32, 32, 32]

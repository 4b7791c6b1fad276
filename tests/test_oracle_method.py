"""Pins for oracle/sketch_sum.py: the method checked against what the paper and
the mathematics fix, never against itself.

  sizes      Eq. heuristic_formula / Eq. sketch_condition, by hand and by brute force
  T1         structured sketch = dense unfolding x explicit Kron/KRP Omega (Eqs. KRP_sketch,
             Kron operator, Prop. 1) on tiny inputs
  T2         QR basis: orthonormal, spans Y, R upper triangular with diag >= 0
  ST-HOSVD   exact multilinear rank recovered; rank rule on a closed-form spectrum
  T3         target >= sum of term ranks => recompression equals the dense sum (Sec. 3.3);
             Sec. 5.1.1 shared-subspace construction recovers rank 10
  T4         shared factors => one Tucker tensor with summed cores; permutation
             invariance; homogeneity
  T5         Sec. 5.1.2 cancellation: the sum equals X_target
  T8         gradient with Q fixed vs central finite differences (exact for a quadratic)
"""
import math

import numpy as np
import pytest

from oracle import rng
from oracle import sketch_sum as ss
from oracle.tensor import (khatri_rao, kron, multi_ttm, tucker_full, tucker_sum_full, unfold)
from paper_2603_13532_gb300 import workloads as wl


def _rand_terms(rng_, dims, ranks_list):
    return [(rng_.standard_normal(r), [rng_.standard_normal((n, rm)) for n, rm in zip(dims, r)])
            for r in ranks_list]


# ------------------------------------------------------------------ sizes
def test_sketch_sizes_worked_values():
    # Kron, d=3, ell=32: (32 s)^2 >= 32^3 -> s = 6 (ceil(181.02/32)); S_n = 36
    assert ss.sketch_sizes("kron", [32, 32, 32]) == ([6, 6, 6], [36, 36, 36])
    # Kron, d=4, ell=48: s^3 >= 48 -> s = 4; S_n = 64
    assert ss.sketch_sizes("kron", [48] * 4) == ([4] * 4, [64] * 4)
    # KRP: s = max ell
    assert ss.sketch_sizes("krp", [58, 40, 51]) == ([58] * 3, [58] * 3)
    # ell = (4,4,4): (prod ell)^(1/2) = 8 exactly, s = 2 (a float root may land at 2.0000001)
    assert ss.kron_sketch_sizes([4, 4, 4]) == [2, 2, 2]


@pytest.mark.parametrize("ell", [[3, 5, 7], [10, 2, 9, 4], [1, 1], [17, 4], [6, 6, 6, 6, 6]])
def test_kron_sizes_satisfy_condition_and_heuristic(ell):
    d = len(ell)
    s = ss.kron_sketch_sizes(ell)
    for n in range(d):
        assert math.prod(s[j] for j in range(d) if j != n) >= ell[n]      # Eq. sketch_condition
    C = math.prod(ell) ** (1.0 / (d - 1))
    for si, li in zip(s, ell):
        # the integer form equals ceil(C / ell_i) whenever C / ell_i is not within 1e-9 of an integer
        x = C / li
        if abs(x - round(x)) > 1e-9:
            assert si == math.ceil(x)


# ------------------------------------------------------------------ T1
def _explicit_sketch(kind, omegas, n):
    others = [omegas[j] for j in reversed(range(len(omegas))) if j != n]
    return khatri_rao(*others) if kind == "krp" else kron(*others)


@pytest.mark.parametrize("kind", ["krp", "kron"])
@pytest.mark.parametrize("dims,ranks_list,ell", [
    ([5, 6, 7], [(2, 3, 2), (3, 1, 2), (1, 2, 3)], [4, 3, 5]),
    ([4, 3, 5, 4], [(2, 2, 3, 1), (1, 3, 2, 2)], [3, 2, 4, 3]),
])
def test_T1_structured_sketch_equals_dense_bruteforce(kind, dims, ranks_list, ell):
    g = np.random.default_rng(3)
    terms = _rand_terms(g, dims, ranks_list)
    X = tucker_sum_full(terms)
    cols, S = ss.sketch_sizes(kind, ell)
    omegas = ss.draw_omegas(9, 0, dims, cols)
    Ys, Ms, Vs = ss.sketch_sum(terms, omegas, kind)
    for n in range(len(dims)):
        Sn = _explicit_sketch(kind, omegas, n)
        assert Sn.shape == (X.size // dims[n], S[n])
        ref = unfold(X, n) @ Sn
        assert np.linalg.norm(Ys[n] - ref) <= 1e-13 * np.linalg.norm(ref)
        # stage (a) is the plain product U^T Omega for every term
        for k, (_, Us) in enumerate(terms):
            np.testing.assert_allclose(Ms[k][n], Us[n].T @ omegas[n], rtol=1e-14, atol=1e-14)


# ------------------------------------------------------------------ T2
def test_T2_orthonormal_basis():
    g = np.random.default_rng(4)
    Y = g.standard_normal((40, 7)) @ np.diag(10.0 ** -np.arange(7))
    Q = ss.orthonormal_basis(Y)
    np.testing.assert_allclose(Q.T @ Q, np.eye(7), atol=1e-14)
    R = Q.T @ Y
    assert np.allclose(np.tril(R, -1), 0, atol=1e-13)
    assert np.all(np.diag(R) >= 0)
    np.testing.assert_allclose(Q @ R, Y, atol=1e-13)
    # classical Gram-Schmidt by hand on a well-conditioned Y gives the same unique factor
    Y2 = g.standard_normal((12, 4))
    Q2 = ss.orthonormal_basis(Y2)
    cols = []
    for j in range(4):
        v = Y2[:, j].copy()
        for q in cols:
            v -= (q @ Y2[:, j]) * q
        cols.append(v / np.linalg.norm(v))
    np.testing.assert_allclose(Q2, np.stack(cols, axis=1), atol=1e-12)


# ------------------------------------------------------------------ ST-HOSVD
def test_st_hosvd_recovers_exact_multilinear_rank():
    g = np.random.default_rng(5)
    G, Us = g.standard_normal((3, 2, 4)), [np.linalg.qr(g.standard_normal((n, r)))[0]
                                            for n, r in zip((8, 7, 9), (3, 2, 4))]
    X = tucker_full(G, Us)
    core, Ps, ranks, svs = ss.st_hosvd(X, tol=1e-12)
    assert ranks == [3, 2, 4]
    np.testing.assert_allclose(tucker_full(core, Ps), X, atol=1e-13)
    # singular values of the first unfolding = sqrt of the Gram eigenvalues (a different routine)
    ev = np.sort(np.linalg.eigvalsh(unfold(X, 0) @ unfold(X, 0).T))[::-1]
    np.testing.assert_allclose(svs[0][:3], np.sqrt(ev[:3]), rtol=1e-12)


def test_st_hosvd_rank_rule_closed_form():
    # superdiagonal core with entries 1, 1e-1, ..., 1e-5: every unfolding has exactly those
    # singular values; theta = tol^2 ||H||^2 / d picks the rank by the tail rule of Alg. 2
    vals = 10.0 ** -np.arange(6)
    H = np.zeros((6, 6, 6))
    for i, v in enumerate(vals):
        H[i, i, i] = v
    norm2 = float(np.sum(vals ** 2))
    for tol in [1e-1, 1e-3, 0.7e-2]:
        theta = tol ** 2 * norm2 / 3
        r_expect = min(r for r in range(1, 7) if np.sum(vals[r:] ** 2) <= theta)
        _, _, ranks, _ = ss.st_hosvd(H, tol=tol)
        assert ranks == [r_expect] * 3
    _, _, ranks, _ = ss.st_hosvd(H, target=[4, 2, 5])
    assert ranks == [4, 2, 5]


def test_truncation_error_estimate_is_the_truncation_error():
    """The discarded parts of the successive ST-HOSVD modes are orthogonal: the estimate from the
    singular values equals ||H - core x_n P_n||_F / ||H||_F computed directly; the superdiagonal
    closed form gives sqrt(sum over modes of the discarded squared diagonal) / ||H||."""
    g = np.random.default_rng(12)
    H = g.standard_normal((9, 7, 8)) * np.logspace(0, -3, 9)[:, None, None]
    for target in ([4, 3, 5], [9, 7, 8], [1, 1, 1]):
        core, Ps, ranks, svs = ss.st_hosvd(H, target=target)
        direct = np.linalg.norm(H - tucker_full(core, Ps)) / np.linalg.norm(H)
        assert abs(ss.truncation_error_estimate(H, svs, ranks) - direct) <= 1e-12 * max(direct, 1.0)
    vals = 10.0 ** -np.arange(6)
    D = np.zeros((6, 6, 6))
    for i, v in enumerate(vals):
        D[i, i, i] = v
    core, Ps, ranks, svs = ss.st_hosvd(D, target=[2, 4, 3])
    # mode 1 drops entries 2..5; after that the core is 2 x 6 x 6 with entries 1, 0.1, so modes 2, 3
    # drop nothing more
    expect = np.sqrt(np.sum(vals[2:] ** 2)) / np.linalg.norm(vals)
    assert abs(ss.truncation_error_estimate(D, svs, ranks) - expect) <= 1e-14


# ------------------------------------------------------------------ T3
def _recon(res):
    return tucker_full(res["core"], res["factors"])


@pytest.mark.parametrize("kind", ["kron", "krp"])
def test_T3_exact_recovery_exact_recovery_workload(kind):
    w = wl.exact_recovery()
    p = w.problems[0]
    res = ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=w.seed)
    if kind == "kron":
        assert res["cols"] == [6, 6, 6] and res["S"] == [36, 36, 36]
    X = tucker_sum_full(p.terms())
    err = np.linalg.norm(_recon(res) - X) / np.linalg.norm(X)
    assert err <= 1e-13, err
    assert all(r <= 32 for r in res["ranks"])


@pytest.mark.parametrize("kind", ["krp", "kron"])
def test_T3_shared_subspace_sec511(kind):
    w = wl.shared_subspace(n=60, K=20, d=4, kind=kind)
    p = w.problems[0]
    res = ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=w.seed, tol=1e-6)
    assert res["ranks"] == [10] * 4
    X = tucker_sum_full(p.terms())
    assert np.linalg.norm(_recon(res) - X) <= 1e-13 * np.linalg.norm(X)


# ------------------------------------------------------------------ T4
def test_T4_shared_factors_equal_summed_core():
    g = np.random.default_rng(6)
    dims, r = [9, 8, 7], (3, 2, 3)
    Us = [g.standard_normal((n, rm)) for n, rm in zip(dims, r)]
    cores = [g.standard_normal(r) for _ in range(4)]
    terms = [(G, Us) for G in cores]
    one = [(sum(cores), Us)]
    a = ss.recompress(terms, "krp", [3, 2, 3], [2, 2, 2], seed=1)
    b = ss.recompress(one, "krp", [3, 2, 3], [2, 2, 2], seed=1)
    for Ya, Yb in zip(a["Y"], b["Y"]):
        np.testing.assert_allclose(Ya, Yb, rtol=1e-13, atol=1e-13 * np.abs(Yb).max())
    np.testing.assert_allclose(_recon(a), _recon(b), atol=1e-13 * np.abs(_recon(b)).max())


def test_T4_permutation_invariance_and_homogeneity():
    g = np.random.default_rng(7)
    dims = [10, 9, 8]
    terms = _rand_terms(g, dims, [(2, 3, 2), (3, 3, 1), (1, 2, 2), (2, 2, 2)])
    X = tucker_sum_full(terms)
    # mode ranks of X: min(8, 10), min(10, 9), min(7, 8) = (8, 9, 7) <= target 9
    base = ss.recompress(terms, "krp", [9, 9, 9], [1, 1, 1], seed=2)
    perm = ss.recompress(terms[::-1], "krp", [9, 9, 9], [1, 1, 1], seed=2)
    for Ya, Yb in zip(base["Y"], perm["Y"]):
        np.testing.assert_allclose(Ya, Yb, atol=1e-12 * np.abs(Ya).max())
    # exact in both orders
    for res in (base, perm):
        assert np.linalg.norm(_recon(res) - X) <= 1e-12 * np.linalg.norm(X)
    scaled = ss.recompress(terms, "krp", [9, 9, 9], [1, 1, 1], seed=2, alpha=[-2.5] * 4)
    np.testing.assert_allclose(_recon(scaled), -2.5 * _recon(base), atol=1e-12 * np.abs(X).max())


def test_T4_term_weights_are_a_weighted_sum():
    g = np.random.default_rng(8)
    dims = [7, 6, 5]
    terms = _rand_terms(g, dims, [(2, 2, 2), (1, 3, 2)])
    alpha = [0.5, -3.0]
    X = 0.5 * tucker_full(*terms[0]) - 3.0 * tucker_full(*terms[1])
    res = ss.recompress(terms, "kron", [5, 5, 4], [1, 1, 1], seed=3, alpha=alpha)
    assert np.linalg.norm(_recon(res) - X) <= 1e-12 * np.linalg.norm(X)


# ------------------------------------------------------------------ T5
@pytest.mark.parametrize("kind", ["krp", "kron"])
def test_T5_cancellation_sec512(kind):
    w = wl.cancellation(n=60, kind=kind)
    p = w.problems[0]
    res = ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=w.seed, tol=1e-6)
    Xt = tucker_full(w.notes["target_core"], w.notes["target_factors"])
    err = np.linalg.norm(_recon(res) - Xt) / np.linalg.norm(Xt)
    # The noise terms (norm ~3.5e6) cancel exactly in exact arithmetic; in float64 even the
    # dense sum of these terms is off by ~1e-9 relative to ||X_target|| ~ 1.4, so the floor is
    # eps * 3.5e6 / 1.4 ~ 3e-10 per rounding, summed over K = 60 terms and d stages.  The paper
    # quotes ~2e-11 for its own draws (Fig. Synthetic_cancellation caption); a dropped or
    # mis-signed term would leave an O(1) to O(1e6) error.
    assert err <= 5e-8, err
    assert res["ranks"] == [5, 5, 5]


# ------------------------------------------------------------------ T8
def test_T8_projection_gradient_central_differences():
    g = np.random.default_rng(9)
    dims = [6, 5, 7]
    terms = _rand_terms(g, dims, [(2, 3, 2), (3, 2, 2)])
    Qs = [np.linalg.qr(g.standard_normal((n, 4)))[0] for n in dims]
    T = g.standard_normal((4, 4, 4))

    def loss(tt):
        H = ss.project_core(tt, Qs)
        return float(np.sum((H - T) ** 2))

    H = ss.project_core(terms, Qs)
    dG, dU = ss.project_core_vjp(terms, Qs, 2.0 * (H - T))
    h = 1e-3
    for k in range(2):
        G, Us = terms[k]
        for idx in [(0, 0, 0), (1, 1, 1), tuple(s - 1 for s in G.shape)]:
            Gp, Gm = G.copy(), G.copy()
            Gp[idx] += h
            Gm[idx] -= h
            tp = [t if i != k else (Gp, Us) for i, t in enumerate(terms)]
            tm = [t if i != k else (Gm, Us) for i, t in enumerate(terms)]
            fd = (loss(tp) - loss(tm)) / (2 * h)
            assert math.isclose(fd, dG[k][idx], rel_tol=1e-8, abs_tol=1e-9)
        for n in range(3):
            for (i, j) in [(0, 0), (dims[n] - 1, Us[n].shape[1] - 1)]:
                Up, Um = [u.copy() for u in Us], [u.copy() for u in Us]
                Up[n][i, j] += h
                Um[n][i, j] -= h
                tp = [t if q != k else (G, Up) for q, t in enumerate(terms)]
                tm = [t if q != k else (G, Um) for q, t in enumerate(terms)]
                fd = (loss(tp) - loss(tm)) / (2 * h)
                assert math.isclose(fd, dU[k][n][i, j], rel_tol=1e-8, abs_tol=1e-9)


def test_projection_is_linear_in_terms():
    g = np.random.default_rng(10)
    dims = [6, 6, 6]
    terms = _rand_terms(g, dims, [(2, 2, 2), (3, 1, 2), (2, 3, 3)])
    Qs = [np.linalg.qr(g.standard_normal((6, 3)))[0] for _ in dims]
    H = ss.project_core(terms, Qs)
    parts = sum(ss.project_core([t], Qs) for t in terms)
    np.testing.assert_allclose(H, parts, atol=1e-14)
    X = tucker_sum_full(terms)
    np.testing.assert_allclose(H, multi_ttm(X, [Q.T for Q in Qs]), atol=1e-13)

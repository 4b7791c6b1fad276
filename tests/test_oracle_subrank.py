"""Pins for oracle/subrank.py (Alg. 5): the heuristic checked against what the
mathematics fixes, never against itself.

  closed form   factors in mutually orthogonal column blocks: B_n is diagonal with
                eigenvalues ||G_k||^2 (multiplicity r_kn); the effective ranks for
                several eps worked out by hand, including values that tell the
                order d from the number of terms K and ||G|| from ||G||^2
  library       eig(V^T V) = squared singular values of V (numpy SVD of V built here)
  shared basis  U_k^(n) = U for all k: one eigenvalue sum_k ||G_k||^2 of multiplicity r
  invariants    scaling all cores, rotating a mode's factors, permuting terms
"""
import math

import numpy as np
import pytest

from oracle import subrank as sr
from paper_2603_13532_gb300 import workloads as wl


def _block_terms(seed, n, ranks_per_term, weights):
    """Terms whose mode-m factors are disjoint column blocks of one Haar matrix per mode and
    whose cores have Frobenius norm weights[k] exactly."""
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


# mode-0 ranks (3, 2, 2, 5) with weights (4, 2, 1, 1e-4): eigenvalues 16 x3, 4 x2, 1 x2, 1e-8 x5,
# trace 58.00000005.  Modes 1 and 2 use other ranks so every mode has its own spectrum.
RANKS = [(3, 4, 1), (2, 1, 5), (2, 2, 2), (5, 3, 1)]
WEIGHTS = [4.0, 2.0, 1.0, 1e-4]


def test_closed_form_spectrum():
    terms = _block_terms(1, 40, RANKS, WEIGHTS)
    lam = sr.spectrum(terms, 0)
    expect = np.array([16.0] * 3 + [4.0] * 2 + [1.0] * 2 + [1e-8] * 5)
    np.testing.assert_allclose(lam, expect, rtol=1e-12, atol=1e-14)
    # mode 1: ranks (4, 1, 2, 3) -> 16 x4, 4, 1 x2, 1e-8 x3
    expect1 = np.array([16.0] * 4 + [4.0] + [1.0] * 2 + [1e-8] * 3)
    np.testing.assert_allclose(sr.spectrum(terms, 1), expect1, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("eps,rank0", [
    # tau = eps^2 / 3 * 58.00000005
    (2.0, 1),        # tau = 77.3 >= trace: every r qualifies, r = 1
    (0.35, 5),       # tau = 2.368: tail(5) = 2.00000005 <= tau < tail(4) = 6.00000005
                     # (eps^2 / K with K = 4 would give 1.776 and rank 6; weights ||G||^2
                     #  instead of ||G|| would give eigenvalues 256, 16, 1, 1e-16 and rank 4)
    (0.3, 6),        # tau = 1.74: tail(6) = 1.00000005 <= tau < tail(5)
    (1e-3, 7),       # tau = 1.93e-5: tail(7) = 5e-8 <= tau < tail(6) = 1.00000005
    (1e-6, 12),      # tau = 1.93e-11 < 1e-8: nothing can be dropped
])
def test_closed_form_effective_rank(eps, rank0):
    terms = _block_terms(1, 40, RANKS, WEIGHTS)
    res = sr.effective_subrank(terms, eps, [3, 3, 3], kind="krp")
    assert res["rank"][0] == rank0
    assert res["ell"][0] == rank0 + 3
    assert math.isclose(res["tau"][0], eps * eps / 3 * 58.00000005, rel_tol=1e-12)
    assert res["cols"] == [max(res["ell"])] * 3


def test_alpha_weights_use_the_scaled_cores():
    # alpha = (0.5, -2, 1, 3) turns the weights (4, 2, 1, 1e-4) into (2, 4, 1, 3e-4):
    # mode 0 eigenvalues 4 x3, 16 x2, 1 x2, 9e-8 x5; trace 12 + 32 + 2 + 4.5e-7 = 46.00000045
    terms = _block_terms(1, 40, RANKS, WEIGHTS)
    res = sr.effective_subrank(terms, 0.3, [0, 0, 0], alpha=[0.5, -2.0, 1.0, 3.0])
    expect = np.array([16.0] * 2 + [4.0] * 3 + [1.0] * 2 + [9e-8] * 5)
    np.testing.assert_allclose(res["lam"][0], expect, rtol=1e-12, atol=1e-14)
    # tau = 0.03 * 46.00000045 = 1.38: tail(6) = 1.00000045 <= tau < tail(5) = 2.00000045
    assert res["rank"][0] == 6


def test_spectrum_is_squared_singular_values():
    rng = np.random.default_rng(7)
    n, d = 30, 3
    terms = []
    for k in range(5):
        r = [int(x) for x in rng.integers(2, 9, size=d)]
        terms.append((rng.standard_normal(r) * (k + 1), [rng.standard_normal((n, rm)) for rm in r]))
    for m in range(d):
        V = np.hstack([np.linalg.norm(G.ravel()) * Us[m] for G, Us in terms])
        sv = np.linalg.svd(V, compute_uv=False)
        lam = sr.spectrum(terms, m)
        assert len(lam) == V.shape[1]
        expect = np.zeros(V.shape[1])
        expect[:len(sv)] = sv ** 2
        np.testing.assert_allclose(lam, expect, rtol=0, atol=1e-11 * expect[0])


def test_shared_factors_give_one_eigenvalue():
    rng = np.random.default_rng(3)
    n, r, K = 50, 6, 7
    Us = [wl.haar(rng, n, r) for _ in range(3)]
    terms = [(rng.standard_normal((r, r, r)), Us) for _ in range(K)]
    total = sum(float(np.sum(G * G)) for G, _ in terms)
    for m in range(3):
        lam = sr.spectrum(terms, m)
        np.testing.assert_allclose(lam[:r], total, rtol=1e-12)
        assert np.all(lam[r:] <= 1e-12 * total)
    res = sr.effective_subrank(terms, 1e-6, [2, 2, 2])
    assert res["rank"] == [r] * 3 and res["ell"] == [r + 2] * 3


def test_invariants():
    rng = np.random.default_rng(11)
    n, d = 24, 3
    terms = []
    for k in range(6):
        r = [int(x) for x in rng.integers(2, 7, size=d)]
        G = rng.standard_normal(r) * 10.0 ** (-k)
        terms.append((G, [rng.standard_normal((n, rm)) for rm in r]))
    base = sr.effective_subrank(terms, 1e-4, [1, 2, 3])
    scaled = sr.effective_subrank([(7.5 * G, Us) for G, Us in terms], 1e-4, [1, 2, 3])
    assert scaled["rank"] == base["rank"]
    Qr = wl.haar(rng, n, n)
    rotated = sr.effective_subrank([(G, [Qr @ Us[0]] + Us[1:]) for G, Us in terms], 1e-4, [1, 2, 3])
    assert rotated["rank"] == base["rank"]
    np.testing.assert_allclose(rotated["lam"][0], base["lam"][0], rtol=0, atol=1e-12 * base["lam"][0][0])
    permuted = sr.effective_subrank(terms[::-1], 1e-4, [1, 2, 3])
    assert permuted["rank"] == base["rank"]
    # the ranks never exceed min(n, R_n) and shrink as eps grows
    loose = sr.effective_subrank(terms, 1e-1, [0, 0, 0])
    for m in range(d):
        R = sum(U[m].shape[1] for _, U in terms)
        assert 1 <= loose["rank"][m] <= base["rank"][m] <= min(n, R)

"""Effective subrank heuristic (Alg. 5, Sec. 3.2 "Heuristic Subrank Selection").

TEST INFRASTRUCTURE ONLY: see ``oracle/__init__.py``.

Phase 1, for every mode n of a sum of K Tucker terms [[G_k; U_k^(1), ..., U_k^(d)]]:
  V_n = [ ||G_1||_F U_1^(n), ..., ||G_K||_F U_K^(n) ]     energy-weighted concatenation
  B_n = V_n^T V_n
  lambda = eig(B_n), clamped at zero and sorted in descending order
  tau = eps^2 / d * sum_j lambda_j
  rt_n = min{ r >= 1 : sum_{j > r} lambda_j <= tau }
  ell_n = rt_n + p_n
Phase 2: the sketch sizes from ell (Eq. heuristic_formula for Kronecker, s = max ell
for Khatri-Rao), as ``sketch_sum.sketch_sizes``.

Readings:
* the paper's d (number of summands) is K here and its N (the order) is d, so the
  threshold is eps^2 / d (the order) times the eigenvalue sum;
* with term weights alpha_k the k-th summand's core is alpha_k G_k, so its weight is
  |alpha_k| ||G_k||_F (the sign cannot change an eigenvalue of B_n);
* eigenvalues come from LAPACK's symmetric solver on B_n in float64, exactly the
  R_n x R_n matrix of the algorithm.
"""
import numpy as np

from .sketch_sum import scaled_terms, sketch_sizes


def term_weights(terms):
    """||G_k||_F of every term (the weights of the concatenation V_n)."""
    return np.array([np.sqrt(np.sum(np.asarray(G, dtype=np.float64) ** 2)) for G, _ in terms])


def weighted_concatenation(terms, n):
    """V_n = [||G_1||_F U_1^(n), ..., ||G_K||_F U_K^(n)] (n_n x R_n)."""
    w = term_weights(terms)
    return np.concatenate([wk * np.asarray(Us[n], dtype=np.float64) for wk, (_, Us) in zip(w, terms)],
                          axis=1)


def weighted_gram(terms, n):
    """B_n = V_n^T V_n (R_n x R_n)."""
    V = weighted_concatenation(terms, n)
    return V.T @ V


def spectrum(terms, n):
    """sort(max(0, eig(B_n)), 'descend')."""
    lam = np.linalg.eigvalsh(weighted_gram(terms, n))
    return np.sort(np.maximum(lam, 0.0))[::-1]


def effective_rank(lam, eps, order):
    """min{r >= 1 : sum_{j > r} lambda_j <= eps^2 / order * sum_j lambda_j}, lambda descending."""
    lam = np.asarray(lam, dtype=np.float64)
    tau = eps * eps / order * float(np.sum(lam))
    for r in range(1, len(lam) + 1):
        if float(np.sum(lam[r:])) <= tau:
            return r
    return len(lam)


def effective_subrank(terms, eps, oversampling, kind="krp", alpha=None):
    """Alg. 5: effective ranks rt_n, ell_n = rt_n + p_n and the sketch sizes.

    Returns a dict with ``rank`` (rt_n), ``ell``, ``cols`` (columns of Omega_j), ``S``
    (columns of Y_n), ``lam`` (per-mode spectra, descending) and ``tau`` (per mode).
    """
    terms = scaled_terms(terms, alpha)
    d = len(terms[0][1])
    lams, ranks, taus = [], [], []
    for n in range(d):
        lam = spectrum(terms, n)
        lams.append(lam)
        taus.append(eps * eps / d * float(np.sum(lam)))
        ranks.append(effective_rank(lam, eps, d))
    ell = [r + p for r, p in zip(ranks, oversampling)]
    cols, S = sketch_sizes(kind, ell)
    return dict(rank=ranks, ell=ell, cols=cols, S=S, lam=lams, tau=taus)

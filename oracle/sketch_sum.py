"""Sketching-based summation of Tucker tensors (KronSum-Tucker, Alg. 3; KRPSum-Tucker, Alg. 4).

TEST INFRASTRUCTURE ONLY: see ``oracle/__init__.py``.

A problem is a list of K Tucker terms X^(k) = [[G_k; U_k^(1), ..., U_k^(d)]]
(``terms = [(G_k, [U_k1, ..., U_kd]), ...]``) plus optional term weights
alpha_k (TuckerAxby scales the cores, Alg. 1).  Everything is float64 and
follows the paper's stages in order:

  stage 1  sketch sizes from ell_n = target_n + p_n (Eq. heuristic_formula for
           Kronecker, s = max ell for Khatri-Rao, Sec. 3.2)
  stage 2  Omega_j, M_kj = U_kj^T Omega_j, the structured sketches
           Y_n = sum_k U_kn V_kn (Eqs. KRP_sketch_unfolding, Kron_sketch_unfolding)
           and an orthonormal basis Q_n = qr(Y_n, 'econ')
  stage 3  H = sum_k G_k x_1 (Q_1^T U_k1) ... x_d (Q_d^T U_kd) (eq. after Sec. 3.3's
           core projection paragraph)
  stage 4  ST-HOSVD(H) (Alg. 2, phase 2), U~_n = Q_n P_n

Readings where the paper is silent or inconsistent:
* the paper's d (number of summands) is K here and its N (order) is d;
* effective ranks: ell_n = target_rank_n + oversampling_n replaces Alg. 5
  phase 1; the final truncation keeps min(target_n, columns of Q_n), or the
  tolerance rule of Alg. 2 when ``tol > 0`` (then capped by the target);
* Kronecker sizes use the exact integer form of Eq. heuristic_formula,
  s_i = min{s >= 1 : (s ell_i)^(d-1) >= prod_j ell_j};
* Q_n is made unique by requiring diag(R) >= 0;
* Alg. 3 returns U_n where U~_n = Q_n V_n is meant.
"""
import math

import numpy as np

from . import rng
from .tensor import khatri_rao, multi_ttm, ttm, unfold


# ---------------------------------------------------------------- stage 1
def kron_sketch_sizes(ell):
    """Per-mode Kronecker sketch sizes s_i (Eq. heuristic_formula, integer form).

    s_i = ceil((prod_j ell_j)^(1/(d-1)) / ell_i) equals the least s with
    (s ell_i)^(d-1) >= prod_j ell_j; the integer form avoids a floating point
    root landing just above an integer.
    """
    d = len(ell)
    if d < 2:
        raise ValueError("order must be at least 2")
    P = math.prod(ell)
    sizes = []
    for li in ell:
        s = 1
        while (s * li) ** (d - 1) < P:
            s += 1
        sizes.append(s)
    return sizes


def sketch_sizes(kind, ell):
    """(columns of Omega_j per mode, columns S_n of Y_n per mode).

    Khatri-Rao (Sec. 3.2): s = max_n ell_n for every mode and S_n = s.
    Kronecker (Eq. heuristic_formula): s_j per mode and S_n = prod_{j != n} s_j,
    which satisfies Eq. sketch_condition S_n >= ell_n.
    """
    d = len(ell)
    if kind == "krp":
        s = max(ell)
        return [s] * d, [s] * d
    if kind == "kron":
        s = kron_sketch_sizes(ell)
        return s, [math.prod(s[j] for j in range(d) if j != n) for n in range(d)]
    raise ValueError(f"unknown sketch kind {kind!r}")


# ---------------------------------------------------------------- stage 2
def draw_omegas(seed, problem, dims, cols, rounding=None):
    """Gaussian Omega_j in R^{n_j x s_j}, one per mode (Alg. 3/4 stage 2; factor reuse)."""
    return [rng.omega(seed, problem, j, n, s, rounding) for j, (n, s) in enumerate(zip(dims, cols))]


def factor_sketch(U, Om):
    """M = U^T Omega in R^{r x s} (Sec. 3.1.1 and 3.1.2)."""
    return U.T @ Om


def core_sketch_krp(G, Ms, n):
    """V_(n) = G_(n) (M_d krp ... krp M_{n+1} krp M_{n-1} krp ... krp M_1) (Eq. krp_sketch_result)."""
    others = [Ms[j] for j in reversed(range(len(Ms))) if j != n]
    return unfold(G, n) @ khatri_rao(*others)


def core_sketch_kron(G, Ms, n):
    """V = G x_{j != n} M_j^T, unfolded along n (Alg. 3 inner loop; Eq. kron_sketch_result)."""
    V = G
    for j, M in enumerate(Ms):
        if j != n:
            V = ttm(V, M.T, j)
    return unfold(V, n)


def sketch_sum(terms, omegas, kind):
    """Y_n = sum_k U_kn V_kn for every mode n (Eqs. KRP_sketch_unfolding / Kron_sketch_unfolding).

    Returns (Y, M, V) with M[k][j] = U_kj^T Omega_j and V[k][n] the core sketches.
    """
    d = len(omegas)
    core_sketch = core_sketch_krp if kind == "krp" else core_sketch_kron
    Ms = [[factor_sketch(Us[j], omegas[j]) for j in range(d)] for _, Us in terms]
    Vs = [[core_sketch(G, Ms[k], n) for n in range(d)] for k, (G, _) in enumerate(terms)]
    Ys = []
    for n in range(d):
        Y = np.zeros((terms[0][1][n].shape[0], Vs[0][n].shape[1]))
        for k, (_, Us) in enumerate(terms):
            Y = Y + Us[n] @ Vs[k][n]
        Ys.append(Y)
    return Ys, Ms, Vs


def orthonormal_basis(Y):
    """Q from the economy QR of Y (Householder, LAPACK), columns signed so diag(R) >= 0."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    sign = np.where(np.diag(R) < 0, -1.0, 1.0)
    return Q * sign[None, :]


# ---------------------------------------------------------------- stage 3
def project_core(terms, Qs):
    """H = sum_k G_k x_1 (Q_1^T U_k1) x_2 ... x_d (Q_d^T U_kd) (core projection, Sec. 3.3)."""
    H = None
    for G, Us in terms:
        V = multi_ttm(G, [Q.T @ U for Q, U in zip(Qs, Us)])
        H = V if H is None else H + V
    return H


def project_core_vjp(terms, Qs, Hbar):
    """Gradients of <Hbar, H(G, U; Q)> with Q held fixed (stop-gradient through Q).

    H_(n) = sum_k A_kn G_k,(n) (kron_{j != n} A_kj)^T with A_kj = Q_j^T U_kj, so
    dL/dG_k = Hbar x_1 A_k1^T ... x_d A_kd^T and
    dL/dU_kn = Q_n [ (Hbar x_{j != n} A_kj^T)_(n) G_k,(n)^T ].
    """
    dG, dU = [], []
    d = len(Qs)
    for G, Us in terms:
        A = [Q.T @ U for Q, U in zip(Qs, Us)]
        dG.append(multi_ttm(Hbar, [a.T for a in A]))
        row = []
        for n in range(d):
            W = multi_ttm(Hbar, [a.T for a in A], skip=n)
            row.append(Qs[n] @ (unfold(W, n) @ unfold(G, n).T))
        dU.append(row)
    return dG, dU


# ---------------------------------------------------------------- stage 4
def tail_rank(sv, theta):
    """min{r >= 1 : sum_{j > r} sv_j^2 <= theta} (Alg. 2, rank rule)."""
    sq = np.asarray(sv, dtype=np.float64) ** 2
    for r in range(1, len(sq) + 1):
        if sq[r:].sum() <= theta:
            return r
    return len(sq)


def st_hosvd(H, target=None, tol=0.0):
    """Sequentially truncated HOSVD of H over modes 1..d in order (Alg. 2, phase 2).

    Returns (core, [P_n], ranks, [singular values of each processed unfolding]).
    With ``tol > 0`` the rank rule uses theta = tol^2 ||H||_F^2 / d computed once
    before the loop (Alg. 2); otherwise r_n = min(target_n, rows of H_(n)).
    """
    d = H.ndim
    theta = tol * tol * float(np.sum(H * H)) / d
    Ps, ranks, svs = [], [], []
    for n in range(d):
        L, sv, _ = np.linalg.svd(unfold(H, n), full_matrices=False)
        if tol > 0:
            r = tail_rank(sv, theta)
            if target is not None:
                r = min(r, target[n])
        else:
            r = min(target[n], len(sv))
        P = L[:, :r]
        H = ttm(H, P.T, n)
        Ps.append(P)
        ranks.append(r)
        svs.append(sv)
    return H, Ps, ranks, svs


def truncation_error_estimate(H, svs, ranks):
    """||H - H~||_F / ||H||_F of the ST-HOSVD truncation (Alg. 2, phase 2) from the singular values of
    each processed unfolding: the parts discarded at the successive modes are orthogonal, so the
    squared error is the sum over modes of the discarded squared singular values."""
    tail = sum(float(np.sum(np.asarray(sv, dtype=np.float64)[r:] ** 2)) for sv, r in zip(svs, ranks))
    nh = float(np.sum(np.asarray(H, dtype=np.float64) ** 2))
    return float(np.sqrt(tail / nh)) if nh > 0 else 0.0


# ---------------------------------------------------------------- full method
def scaled_terms(terms, alpha=None):
    """Fold term weights into the cores, as TuckerAxby (Alg. 1) scales them."""
    if alpha is None:
        return list(terms)
    return [(a * G, Us) for a, (G, Us) in zip(alpha, terms)]


def recompress(terms, kind, target, oversampling, seed, problem=0, tol=0.0,
               alpha=None, rounding=None, omegas=None, Qs=None):
    """KronSum-Tucker (Alg. 3) or KRPSum-Tucker (Alg. 4) with target ranks.

    ``omegas`` or ``Qs`` may be supplied to isolate stages (the sketch is
    deterministic given Omega and the projection given Q).  Returns a dict of
    every intermediate: ell, cols, S, omegas, M, V, Y, Q, H, core, factors,
    ranks, P, svs.
    """
    terms = scaled_terms(terms, alpha)
    d = len(terms[0][1])
    dims = [U.shape[0] for U in terms[0][1]]
    ell = [t + p for t, p in zip(target, oversampling)]
    cols, S = sketch_sizes(kind, ell)
    if omegas is None:
        omegas = draw_omegas(seed, problem, dims, cols, rounding)
    Ys, Ms, Vs = sketch_sum(terms, omegas, kind)
    if Qs is None:
        Qs = [orthonormal_basis(Y) for Y in Ys]
    H = project_core(terms, Qs)
    core, Ps, ranks, svs = st_hosvd(H, target, tol)
    factors = [Q @ P for Q, P in zip(Qs, Ps)]
    return dict(ell=ell, cols=cols, S=S, dims=dims, d=d, omegas=omegas, M=Ms, V=Vs,
                Y=Ys, Q=Qs, H=H, core=core, factors=factors, ranks=ranks, P=Ps, svs=svs)

"""Tensor primitives of Sec. 2 in float64 (oracle side).

TEST INFRASTRUCTURE ONLY: see ``oracle/__init__.py``.

Conventions (Sec. 2.1):
* Kronecker product (Def. 1): (A kron B)[i p + k, j q + l] = a_ij b_kl (0-based),
  i.e. numpy.kron.
* Khatri-Rao product (Def. 1): column-wise Kronecker product.
* Mode-k unfolding X_(k) (Eq. unfolding_index): rows indexed by i_k, columns by
  the remaining indices with the FIRST remaining mode varying fastest.
* TTM (Sec. 2.1): Y = X x_k A with A in R^{J x n_k} means Y_(k) = A X_(k).
* Tucker tensor [[G; U_1..U_N]] (Eq. TuckerDecompositionModeProd).

Tensors are numpy arrays indexed (i_1, ..., i_N); "column-major" storage means
mode 1 fastest, which is ``order="F"``.
"""
import numpy as np


def kron(*mats):
    """A_1 kron A_2 kron ... (Def. 1, left factor = slowest index)."""
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(out, m)
    return out


def khatri_rao(*mats):
    """A_1 krp A_2 krp ...: column c is kron of the c-th columns (Def. 1)."""
    r = mats[0].shape[1]
    if any(m.shape[1] != r for m in mats):
        raise ValueError("Khatri-Rao factors need equal column counts")
    out = np.ones((1, r))
    for m in mats:
        out = (out[:, None, :] * m[None, :, :]).reshape(-1, r)
    return out


def unfold(X, k):
    """Mode-k unfolding X_(k) in R^{n_k x prod_{m != k} n_m} (Eq. unfolding_index)."""
    return np.moveaxis(X, k, 0).reshape(X.shape[k], -1, order="F")


def fold(Xk, k, shape):
    """Inverse of :func:`unfold`."""
    rest = [shape[m] for m in range(len(shape)) if m != k]
    return np.moveaxis(Xk.reshape([shape[k]] + rest, order="F"), 0, k)


def ttm(X, A, k):
    """Y = X x_k A, i.e. Y_(k) = A X_(k) (Sec. 2.1)."""
    shape = list(X.shape)
    shape[k] = A.shape[0]
    return fold(A @ unfold(X, k), k, shape)


def multi_ttm(X, mats, skip=None):
    """X x_1 A_1 x_2 ... x_N A_N, modes in ascending order; ``skip`` is left alone."""
    for k, A in enumerate(mats):
        if k != skip and A is not None:
            X = ttm(X, A, k)
    return X


def tucker_full(G, Us):
    """Dense tensor of [[G; U_1, ..., U_N]] (Eq. TuckerDecompositionModeProd)."""
    return multi_ttm(G, Us)


def tucker_sum_full(terms):
    """Dense sum of a list of (G, [U_1..U_N]) Tucker terms."""
    return sum(tucker_full(G, Us) for G, Us in terms)


def tucker_inner(A, Us, B, Vs):
    """<[[A; U]], [[B; V]]> = <A, B x_1 (U_1^T V_1) ... x_N (U_N^T V_N)> without densifying."""
    W = multi_ttm(B, [U.T @ V for U, V in zip(Us, Vs)])
    return float(np.vdot(A, W))


def tucker_sum_inner(terms_a, terms_b):
    """<sum_i X_i, sum_j Y_j> from pairwise Tucker inner products."""
    return sum(tucker_inner(Ga, Ua, Gb, Ub) for Ga, Ua in terms_a for Gb, Ub in terms_b)


def tucker_entries(G, Us, idx):
    """Entries of [[G; U]] at the integer index rows ``idx`` (shape (m, N)), one by one."""
    idx = np.asarray(idx)
    out = np.empty(idx.shape[0])
    for t, ii in enumerate(idx):
        W = G
        for k, U in enumerate(Us):
            W = np.tensordot(U[ii[k]], W, axes=(0, 0))
        out[t] = float(W)
    return out

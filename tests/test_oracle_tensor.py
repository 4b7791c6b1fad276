"""Pins for oracle/tensor.py against the elementwise definitions of Sec. 2.

Each primitive is checked against pure-Python loops over the defining index
formula (Def. 1, Eq. unfolding_index, the TTM sum, Eq. TuckerDecompositionElementwise)
and the identities of Prop. 1 on tiny random inputs.
"""
import itertools
import math

import numpy as np

from oracle.tensor import (fold, khatri_rao, kron, multi_ttm, ttm, tucker_entries,
                           tucker_full, tucker_inner, tucker_sum_inner, unfold)

RNG = np.random.default_rng(11)


def test_kron_elementwise_definition():
    A = RNG.standard_normal((2, 3))
    B = RNG.standard_normal((4, 2))
    K = kron(A, B)
    assert K.shape == (8, 6)
    for i, j, k, l in itertools.product(range(2), range(3), range(4), range(2)):
        # (A kron B)_{(i-1)p+k, (j-1)q+l} = a_ij b_kl, written 0-based
        assert K[i * 4 + k, j * 2 + l] == A[i, j] * B[k, l]


def test_khatri_rao_columnwise_kron():
    A = RNG.standard_normal((3, 4))
    B = RNG.standard_normal((2, 4))
    C = RNG.standard_normal((5, 4))
    KR = khatri_rao(A, B, C)
    for c in range(4):
        for i, k, m in itertools.product(range(3), range(2), range(5)):
            assert math.isclose(KR[(i * 2 + k) * 5 + m, c], A[i, c] * B[k, c] * C[m, c],
                                rel_tol=1e-15)


def test_unfolding_index_formula():
    shape = (2, 3, 4, 2)
    X = RNG.standard_normal(shape)
    for k in range(4):
        Xk = unfold(X, k)
        assert Xk.shape == (shape[k], X.size // shape[k])
        for idx in itertools.product(*[range(n) for n in shape]):
            j, stride = 0, 1
            for m in range(4):          # Eq. unfolding_index, 0-based
                if m == k:
                    continue
                j += idx[m] * stride
                stride *= shape[m]
            assert Xk[idx[k], j] == X[idx]
        np.testing.assert_array_equal(fold(Xk, k, shape), X)


def test_ttm_elementwise_sum():
    X = RNG.standard_normal((3, 4, 2))
    A = RNG.standard_normal((5, 4))
    Y = ttm(X, A, 1)
    assert Y.shape == (3, 5, 2)
    for i1, j, i3 in itertools.product(range(3), range(5), range(2)):
        ref = sum(X[i1, i2, i3] * A[j, i2] for i2 in range(4))
        assert math.isclose(Y[i1, j, i3], ref, rel_tol=1e-13, abs_tol=1e-14)


def _tiny_tucker(shape, ranks):
    G = RNG.standard_normal(ranks)
    Us = [RNG.standard_normal((n, r)) for n, r in zip(shape, ranks)]
    return G, Us


def test_tucker_elementwise_definition():
    G, Us = _tiny_tucker((3, 4, 2), (2, 3, 2))
    X = tucker_full(G, Us)
    for i in itertools.product(range(3), range(4), range(2)):
        ref = sum(G[j] * Us[0][i[0], j[0]] * Us[1][i[1], j[1]] * Us[2][i[2], j[2]]
                  for j in itertools.product(range(2), range(3), range(2)))
        assert math.isclose(X[i], ref, rel_tol=1e-12, abs_tol=1e-13)
    idx = np.array([[0, 0, 0], [2, 3, 1], [1, 2, 0]])
    np.testing.assert_allclose(tucker_entries(G, Us, idx), X[tuple(idx.T)], rtol=1e-13)


def test_prop1_unfolding_identity():
    G, Us = _tiny_tucker((3, 4, 2, 3), (2, 2, 2, 3))
    X = tucker_full(G, Us)
    for k in range(4):
        others = [Us[j] for j in reversed(range(4)) if j != k]   # U_N kron ... kron U_1 minus k
        np.testing.assert_allclose(unfold(X, k), Us[k] @ unfold(G, k) @ kron(*others).T,
                                   rtol=1e-12, atol=1e-12)


def test_prop1_mttkrp_and_multi_ttm():
    shape, ranks = (3, 4, 2, 3), (2, 3, 2, 2)
    G, Us = _tiny_tucker(shape, ranks)
    X = tucker_full(G, Us)
    s = 5
    As = [RNG.standard_normal((n, s)) for n in shape]
    Bs = [RNG.standard_normal((4, n)) for n in shape]
    for k in range(4):
        order = [j for j in reversed(range(4)) if j != k]
        lhs = unfold(X, k) @ khatri_rao(*[As[j] for j in order])
        rhs = Us[k] @ unfold(G, k) @ khatri_rao(*[Us[j].T @ As[j] for j in order])
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
        lhs2 = multi_ttm(X, Bs, skip=k)
        rhs2 = ttm(multi_ttm(G, [Bs[j] @ Us[j] for j in range(4)], skip=k), Us[k], k)
        np.testing.assert_allclose(lhs2, rhs2, rtol=1e-12, atol=1e-12)


def test_tucker_inner_products_match_dense():
    G1, U1 = _tiny_tucker((4, 3, 5), (2, 3, 2))
    G2, U2 = _tiny_tucker((4, 3, 5), (3, 1, 2))
    X1, X2 = tucker_full(G1, U1), tucker_full(G2, U2)
    assert math.isclose(tucker_inner(G1, U1, G2, U2), float(np.vdot(X1, X2)), rel_tol=1e-12)
    terms = [(G1, U1), (G2, U2)]
    assert math.isclose(tucker_sum_inner(terms, terms), float(np.vdot(X1 + X2, X1 + X2)),
                        rel_tol=1e-12)

"""Stage-isolated parity of the final ST-HOSVD truncation (Alg. 2 phase 2; stage 4 of Algs. 3/4).

tks_truncate_core takes the oracle's bases Q_n and projected core H, so every difference is the
truncation's own arithmetic.  TKS_FP64 and TKS_MIXED both run it in float64 (TSQR of each unfolding
and a one-sided Jacobi SVD of its triangular factor; TKS_MIXED takes the mode products
float64-accurate on the tensor cores by exact digit products), so both are held to the float64 bound:
the kept subspaces of two backward-stable SVDs differ by eps ||H|| / gap in angle, and the
reconstructions Q P P^T ... by a few eps ||H|| (the spectra here have no near-degenerate gap at the
truncation point).  TKS_MIXED_F32LA runs it in float32: 1e-5.
"""
import numpy as np
import pytest

from oracle import sketch_sum as ss
from oracle.tensor import tucker_full
from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problems(d, seed, bf16):
    g = np.random.default_rng(seed)
    probs = []
    for dims, K in ([[72, 40, 136, 48][:d], 3], [[64, 96, 56, 40][:d], 4], [[128] * d, 6]):
        cores, facs = [], []
        for _ in range(K):
            r = [min(int(x), n) for x, n in zip(g.integers(2, 12, size=d), dims)]
            cores.append(g.standard_normal(r))
            facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
        probs.append(wl.Problem(list(dims), cores, facs, [9] * d, [4] * d, alpha=list(g.standard_normal(K))))
    return wl._finish(probs, True) if bf16 else probs


def _recon(res, r=None):
    return tucker_full(res["core"], res["factors"])


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f32la"])
@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("tol", [0.0, 1e-2])
def test_truncation_of_the_oracle_core(cuda_lib, precision, d, tol):
    from paper_2603_13532_gb300 import binding
    bf16 = precision != "fp64"
    probs = _problems(d, 40 + d, bf16)
    plan = binding.Plan(probs, kind="krp", precision=precision, seed=5, tol=tol)
    refs = [ss.recompress(p.terms(), "krp", p.target, p.oversampling, seed=5, problem=i, alpha=p.alpha, tol=tol,
                          rounding="bf16" if bf16 else None) for i, p in enumerate(probs)]
    outs = plan.truncate([r["Q"] for r in refs], [r["H"] for r in refs])
    bound = 1e-5 if precision == "mixed_f32la" else 1e-12
    for i, (got, ref) in enumerate(zip(outs, refs)):
        assert got["ranks"] == ref["ranks"], (i, got["ranks"], ref["ranks"])
        Xo = _recon(ref)
        Xg = _recon(got)
        err = np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo)
        assert err <= bound, (precision, d, tol, i, err)
        # the factors are orthonormal (columns beyond the kept rank are zero)
        for m, U in enumerate(got["factors"]):
            k = got["ranks"][m]
            G = U[:, :k].T @ U[:, :k]
            assert np.abs(G - np.eye(k)).max() <= (1e-5 if precision == "mixed_f32la" else 1e-12), (m, k)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_truncation_decay512_float64_bound(cuda_lib, precision):
    """The bench workload's spectrum (10^(-i/8) per mode, truncation at 48 of 58): both float64 paths
    reproduce the oracle's truncation of its own H to the float64 bound."""
    bf16 = precision != "fp64"
    w = wl.decay512(bf16=bf16)
    p = w.problems[0]
    from paper_2603_13532_gb300 import binding
    plan = binding.Plan(w.problems, kind=w.kind, precision=precision, seed=w.seed)
    ref = ss.recompress(p.terms(), w.kind, p.target, p.oversampling, seed=w.seed,
                        rounding="bf16" if bf16 else None)
    got = plan.truncate([ref["Q"]], [ref["H"]])[0]
    assert got["ranks"] == ref["ranks"] == [48, 48, 48]
    # compare the truncated cores through the bases: H ~ G x_n P_n, in the coordinates of Q
    Hg = tucker_full(got["core"], [Q.T @ U for Q, U in zip(ref["Q"], got["factors"])])
    Ho = tucker_full(ref["core"], ref["P"])
    err = np.linalg.norm(Hg - Ho) / np.linalg.norm(ref["H"])
    assert err <= 1e-12, err


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f32la"])
@pytest.mark.parametrize("d", [3, 4])
def test_truncation_error_estimate(cuda_lib, precision, d):
    """tks_truncation_error after tks_truncate_core on the oracle's H: the relative error of the
    ST-HOSVD from the discarded singular values, against the oracle's (1e-12 absolute in float64,
    1e-5 with float32 linear algebra), and against ||H - H~|| / ||H|| of the returned truncation."""
    from paper_2603_13532_gb300 import binding
    bf16 = precision != "fp64"
    probs = _problems(d, 60 + d, bf16)
    plan = binding.Plan(probs, kind="krp", precision=precision, seed=9)
    refs = [ss.recompress(p.terms(), "krp", p.target, p.oversampling, seed=9, problem=i, alpha=p.alpha,
                          rounding="bf16" if bf16 else None) for i, p in enumerate(probs)]
    outs = plan.truncate([r["Q"] for r in refs], [r["H"] for r in refs])
    est = plan.truncation_error()
    tol = 1e-5 if precision == "mixed_f32la" else 1e-12
    for i, (got, ref) in enumerate(zip(outs, refs)):
        e_ref = ss.truncation_error_estimate(ref["H"], ref["svs"], ref["ranks"])
        assert abs(est[i] - e_ref) <= tol, (i, est[i], e_ref)
        # the same quantity measured: H~ = H x_n (P_n P_n^T) with P_n = Q_n^T U~_n
        Ps = [Q.T @ U for Q, U in zip(ref["Q"], got["factors"])]
        Ht = tucker_full(got["core"], Ps)
        direct = np.linalg.norm(ref["H"] - Ht) / np.linalg.norm(ref["H"])
        assert abs(est[i] - direct) <= 10 * tol, (i, est[i], direct)

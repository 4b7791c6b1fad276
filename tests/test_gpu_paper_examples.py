"""The paper's synthetic examples at their own sizes, end to end on the GPU.

Sec. 5.1.1 (E1): order 4, n = 4000, 100 rank-1 terms whose factors lie in a shared rank-10
subspace per mode, oversampling 2, tolerance 1e-6, both sketches.  The sum has multilinear rank
(10, 10, 10, 10), so the recompression is exact up to rounding; the paper reports ~4e-15 against
the deterministic baseline.  The 4000^4 tensor is never formed: reconstructions are compared on
sampled entries against the exact sum evaluated term by term.
"""
import numpy as np
import pytest

from oracle import sketch_sum as ss
from oracle.tensor import tucker_entries
from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _sampled(prob, got, nsamp=400, seed=0):
    g = np.random.default_rng(seed)
    idx = np.stack([g.integers(0, n, size=nsamp) for n in prob.dims], axis=1)
    ex = sum(tucker_entries(G, Us, idx) for G, Us in prob.terms())
    eg = tucker_entries(got["core"], got["factors"], idx)
    return eg, ex, idx


@pytest.mark.parametrize("kind", ["krp", "kron"])
def test_e1_shared_subspace_full_size_fp64(cuda_lib, kind):
    from paper_2603_13532_gb300 import binding
    w = wl.shared_subspace(n=4000, K=100, d=4, kind=kind)
    p = w.problems[0]
    got = binding.Plan(w.problems, kind=kind, precision="fp64", seed=w.seed, tol=1e-6).recompress()[0]
    assert got["ranks"] == [10, 10, 10, 10]
    eg, ex, idx = _sampled(p, got)
    rel = np.sqrt(np.mean((eg - ex) ** 2) / np.mean(ex ** 2))
    assert rel <= 1e-12, rel
    # and the oracle's own recompression agrees entrywise
    ref = ss.recompress(p.terms(), kind, p.target, p.oversampling, seed=w.seed, tol=1e-6)
    assert ref["ranks"] == [10, 10, 10, 10]
    eo = tucker_entries(ref["core"], ref["factors"], idx)
    assert np.sqrt(np.mean((eg - eo) ** 2) / np.mean(ex ** 2)) <= 1e-12


@pytest.mark.parametrize("precision", ["mixed", "mixed_f32la"])
def test_e1_shared_subspace_full_size_mixed(cuda_lib, precision):
    """E1's shape on the mixed path.  bf16 rounding of Q_n c would leave the subspace, so each
    rank-1 term takes its mode-n factor from the columns of a shared bf16 basis Q_n (4000 x 10)
    and a bf16 scalar core: the sum still has multilinear rank (10, 10, 10, 10) exactly."""
    from paper_2603_13532_gb300 import binding
    g = np.random.default_rng(20260319)
    n, d, K = 4000, 4, 100
    Qs = [wl.to_bf16_values(wl.haar(g, n, 10)) for _ in range(d)]
    cores, facs = [], []
    for _ in range(K):
        cores.append(wl.to_bf16_values(g.standard_normal((1,) * d)))
        facs.append([Q[:, [int(g.integers(0, 10))]] for Q in Qs])
    p = wl.Problem([n] * d, cores, facs, [10] * d, [2] * d)
    got = binding.Plan([p], kind="krp", precision=precision, seed=5, tol=1e-6).recompress()[0]
    assert all(r <= 10 for r in got["ranks"])
    eg, ex, _ = _sampled(p, got)
    rel = np.sqrt(np.mean((eg - ex) ** 2) / np.mean(ex ** 2))
    # the tensor-core products accumulate over n = 4000 in float32: 250 K-steps of 16 spread over
    # eight partial accumulators, each step rounding once, and in A_n = Q_n^T Ucat_n the products
    # share a sign (U_k lies in the span of Q_n), so each contraction carries up to
    # (n / 128) 2^-24 = 1.9e-6; three of them feed H
    assert rel <= 1e-5, rel

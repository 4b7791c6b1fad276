"""Backward of the core projection (tks_project_core_backward) on the GPU.

Checked three ways, all in float64 with the bases Q held fixed (stop-gradient):
  * against the oracle's analytic gradient (oracle.sketch_sum.project_core_vjp): 1e-12 relative;
  * against central finite differences of L = ||H(G, U; Q) - T||^2 evaluated by the GPU forward:
    L is quadratic in any single entry, so (L(x+h) - L(x-h)) / 2h is exact up to rounding
    (h = 1e-3; bound 1e-8 relative to the largest gradient entry);
  * through torch.autograd (binding.ProjectCore) against the direct backward call.
The grad384 workload (d=3, n=384, K=16 terms of rank 16, bf16-valued inputs) is included.
"""
import numpy as np
import pytest
import torch

from oracle import sketch_sum as ss
from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problems(seed=0):
    g = np.random.default_rng(300 + seed)
    probs = []
    for dims, K in ([[40, 33, 29], 3], [[17, 65, 23], 2]):
        cores, facs = [], []
        for _ in range(K):
            r = [int(x) for x in g.integers(1, 7, size=3)]
            cores.append(g.standard_normal(r))
            facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
        probs.append(wl.Problem(dims, cores, facs, [5, 6, 4], [1, 1, 1], alpha=list(g.standard_normal(K))))
    return probs


def _plan(probs, seed=3):
    from paper_2603_13532_gb300 import binding
    return binding.Plan(probs, kind="krp", precision="fp64", seed=seed)


def _qs_and_targets(plan, probs, seed=0):
    g = np.random.default_rng(seed)
    Qs, Ts = [], []
    for p, pi in zip(probs, plan.pinfo):
        Qs.append([np.linalg.qr(g.standard_normal((p.dims[m], pi.basis_cols[m])))[0] for m in range(3)])
        Ts.append(g.standard_normal([pi.basis_cols[m] for m in range(3)]))
    return Qs, Ts


def test_backward_matches_oracle_vjp(cuda_lib):
    probs = _problems()
    plan = _plan(probs)
    Qs, Ts = _qs_and_targets(plan, probs)
    Hs = plan.project(Qs)
    Hbars = [2.0 * (H - T) for H, T in zip(Hs, Ts)]
    got = plan.backward(Qs, Hbars)
    for p, Q, Hb, (dG, dU) in zip(probs, Qs, Hbars, got):
        terms = ss.scaled_terms(p.terms(), p.alpha)
        rG, rU = ss.project_core_vjp(terms, Q, Hb)
        # the oracle differentiates w.r.t. the scaled core alpha_k G_k: chain rule gives alpha_k
        for k, a in enumerate(p.alpha):
            ref = a * rG[k]
            assert np.linalg.norm(dG[k] - ref) <= 1e-12 * max(np.linalg.norm(ref), 1e-30)
            for n in range(3):
                assert np.linalg.norm(dU[k][n] - rU[k][n]) <= 1e-12 * max(np.linalg.norm(rU[k][n]), 1e-30)


def test_backward_central_differences_through_gpu_forward(cuda_lib):
    probs = _problems(1)[:1]
    plan = _plan(probs)
    Qs, Ts = _qs_and_targets(plan, probs, 1)
    Q = plan.pack_bases(Qs)
    T = plan.pack_core(Ts)

    def loss():
        H = torch.zeros(plan.info.core_elems, dtype=torch.float64, device=plan.device)
        plan.project_raw(Q, H)
        torch.cuda.synchronize()
        return float(((H - T) ** 2).sum())

    Hs = plan.project(Qs)
    (dG, dU), = plan.backward(Qs, [2.0 * (Hs[0] - Ts[0])])
    core_v, fac_v = plan.inputs[0]
    h = 1e-3
    scale = max(max(np.abs(x).max() for x in dG), max(np.abs(u).max() for row in dU for u in row))
    # a few entries of each core (packed, mode-1 fastest) and each factor block
    off = 0
    for k, G in enumerate(probs[0].cores):
        for flat_idx in [0, G.size - 1]:
            idx = np.unravel_index(flat_idx, G.shape, order="F")
            pos = off + flat_idx
            old = float(core_v[pos])
            core_v[pos] = old + h
            lp = loss()
            core_v[pos] = old - h
            lm = loss()
            core_v[pos] = old
            assert abs((lp - lm) / (2 * h) - dG[k][idx]) <= 1e-8 * scale
        off += G.size
    for n in range(3):
        col0 = 0
        for k, G in enumerate(probs[0].cores):
            for (i, j) in [(0, 0), (probs[0].dims[n] - 1, G.shape[n] - 1)]:
                pos = i + probs[0].dims[n] * (col0 + j)
                old = float(fac_v[n][pos])
                fac_v[n][pos] = old + h
                lp = loss()
                fac_v[n][pos] = old - h
                lm = loss()
                fac_v[n][pos] = old
                assert abs((lp - lm) / (2 * h) - dU[k][n][i, j]) <= 1e-8 * scale
            col0 += G.shape[n]


def test_autograd_function_matches_direct_backward(cuda_lib):
    from paper_2603_13532_gb300 import binding
    probs = _problems(2)
    plan = _plan(probs)
    Qs, Ts = _qs_and_targets(plan, probs, 2)
    Q = plan.pack_bases(Qs)
    T = plan.pack_core(Ts)
    x = plan.flat_inputs
    x.requires_grad_(True)
    H = binding.ProjectCore.apply(x, Q, plan)
    L = ((H - T) ** 2).sum()
    (gx,) = torch.autograd.grad(L, [x])
    x.requires_grad_(False)
    direct = plan.backward(Qs, [2.0 * (h - t) for h, t in zip(plan.project(Qs), Ts)])
    g = gx.detach().cpu().numpy()
    base = x.storage_offset()
    for p, (core_v, fac_v), (dG, dU) in zip(probs, plan.inputs, direct):
        o = core_v.storage_offset() - base
        flat_dG = np.concatenate([a.ravel(order="F") for a in dG])
        assert np.allclose(g[o: o + flat_dG.size], flat_dG, rtol=1e-12, atol=1e-12)
        for n in range(3):
            o = fac_v[n].storage_offset() - base
            flat_dU = np.hstack([dU[k][n] for k in range(p.num_terms)]).ravel(order="F")
            assert np.allclose(g[o: o + flat_dU.size], flat_dU, rtol=1e-12, atol=1e-12)


def test_backward_grad384_workload(cuda_lib):
    w = wl.grad384()
    p = w.problems[0]
    plan = _plan(w.problems, w.seed)
    ref = ss.recompress(p.terms(), "krp", p.target, p.oversampling, seed=w.seed)
    Qs = [ref["Q"]]
    T = w.notes["target_tensor"]
    H = plan.project(Qs)[0]
    assert np.linalg.norm(H - ref["H"]) <= 1e-12 * np.linalg.norm(ref["H"])
    (dG, dU), = plan.backward(Qs, [2.0 * (H - T)])
    rG, rU = ss.project_core_vjp(p.terms(), ref["Q"], 2.0 * (ref["H"] - T))
    for k in range(p.num_terms):
        assert np.linalg.norm(dG[k] - rG[k]) <= 1e-12 * np.linalg.norm(rG[k])
        for n in range(3):
            assert np.linalg.norm(dU[k][n] - rU[k][n]) <= 1e-12 * np.linalg.norm(rU[k][n])


def test_backward_rejects_order4_plans(cuda_lib):
    from paper_2603_13532_gb300 import binding
    g = np.random.default_rng(9)
    dims = [16, 24, 32, 8]
    prob = wl._finish([wl.Problem(dims, [g.standard_normal((2, 2, 2, 2))],
                                  [[g.standard_normal((n, 2)) for n in dims]], [3, 3, 3, 3], [1, 1, 1, 1])], True)
    plan = binding.Plan(prob, kind="krp", precision="mixed", seed=1)
    Q = torch.zeros(plan.info.basis_elems, dtype=torch.float64, device="cuda")
    Hb = torch.zeros(plan.info.core_elems, dtype=torch.float64, device="cuda")
    dc = torch.zeros(max(1, plan.info.grad_core_elems), dtype=torch.float64, device="cuda")
    df = torch.zeros(max(1, plan.info.grad_factor_elems), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.TksError) as e:
        plan.backward_raw(Q, Hb, dc, df)
    assert e.value.code == 7


# ---------------------------------------------------------------------------------------------------
# Mixed precision (config 5: bf16 factors and cores, float32 accumulation).  The tensor-core products
# take float64 Q and Hbar as three bf16 planes each (about 2^-24 relative) and accumulate in float32
# over K <= 64; the per-term contractions run in float32 over at most r^2 = 256 terms.  Each step adds
# a few units of 2^-24 of its operands' scale, so 1e-5 of each gradient tensor's norm is a bound with
# an order of magnitude to spare, and a dropped term, a wrong offset or a transposed operand fails it
# by orders of magnitude.
def _mixed_problems(seed=0):
    g = np.random.default_rng(500 + seed)
    probs = []
    for dims, K in ([[40, 56, 24], 3], [[64, 16, 48], 2]):
        cores, facs = [], []
        for _ in range(K):
            r = [int(x) for x in g.integers(1, 9, size=3)]
            cores.append(g.standard_normal(r))
            facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
        probs.append(wl.Problem(dims, cores, facs, [5, 7, 6], [2, 1, 3], alpha=list(g.standard_normal(K))))
    return wl._finish(probs, True)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def test_backward_mixed_matches_oracle_vjp(cuda_lib):
    from paper_2603_13532_gb300 import binding
    probs = _mixed_problems()
    plan = binding.Plan(probs, kind="krp", precision="mixed", seed=3)
    Qs, Ts = _qs_and_targets(plan, probs)
    Hbars = [2.0 * (ss.project_core(ss.scaled_terms(p.terms(), p.alpha), Q) - T)
             for p, Q, T in zip(probs, Qs, Ts)]
    got = plan.backward(Qs, Hbars)
    for p, Q, Hb, (dG, dU) in zip(probs, Qs, Hbars, got):
        terms = ss.scaled_terms(p.terms(), p.alpha)
        rG, rU = ss.project_core_vjp(terms, Q, Hb)
        for k, a in enumerate(p.alpha):
            assert _rel(dG[k], a * rG[k]) <= 1e-5, (k, _rel(dG[k], a * rG[k]))
            for n in range(3):
                assert _rel(dU[k][n], rU[k][n]) <= 1e-5, (k, n, _rel(dU[k][n], rU[k][n]))


def test_backward_mixed_grad384_matches_oracle_and_central_differences(cuda_lib):
    """Config 5 at full size on the mixed path: against the oracle's float64 gradient (1e-5 of each
    tensor's norm), and entries against float64 central differences of L = ||H - T||^2 evaluated by the
    float64 GPU forward (exact for a quadratic up to rounding; h = 1e-3)."""
    from paper_2603_13532_gb300 import binding
    w = wl.grad384()
    p = w.problems[0]
    ref = ss.recompress(p.terms(), "krp", p.target, p.oversampling, seed=w.seed)
    T = w.notes["target_tensor"]
    Hbar = 2.0 * (ref["H"] - T)
    mixed = binding.Plan(w.problems, kind="krp", precision="mixed", seed=w.seed)
    (dG, dU), = mixed.backward([ref["Q"]], [Hbar])
    rG, rU = ss.project_core_vjp(p.terms(), ref["Q"], Hbar)
    for k in range(p.num_terms):
        assert _rel(dG[k], rG[k]) <= 1e-5, (k, _rel(dG[k], rG[k]))
        for n in range(3):
            assert _rel(dU[k][n], rU[k][n]) <= 1e-5, (k, n, _rel(dU[k][n], rU[k][n]))
    plan = _plan(w.problems, w.seed)
    Q = plan.pack_bases([ref["Q"]])
    Tt = plan.pack_core([T])

    def loss():
        H = torch.zeros(plan.info.core_elems, dtype=torch.float64, device=plan.device)
        plan.project_raw(Q, H)
        torch.cuda.synchronize()
        return float(((H - Tt) ** 2).sum())

    core_v, fac_v = plan.inputs[0]
    h = 1e-3
    scale = max(max(np.abs(x).max() for x in dG), max(np.abs(u).max() for row in dU for u in row))
    G0 = p.cores[0]
    for flat_idx in [0, 7, G0.size - 1]:
        idx = np.unravel_index(flat_idx, G0.shape, order="F")
        old = float(core_v[flat_idx])
        core_v[flat_idx] = old + h
        lp = loss()
        core_v[flat_idx] = old - h
        lm = loss()
        core_v[flat_idx] = old
        assert abs((lp - lm) / (2 * h) - dG[0][idx]) <= 1e-5 * scale
    for n in range(3):
        for (i, j) in [(0, 0), (p.dims[n] - 1, 3)]:
            old = float(fac_v[n][i + p.dims[n] * j])
            fac_v[n][i + p.dims[n] * j] = old + h
            lp = loss()
            fac_v[n][i + p.dims[n] * j] = old - h
            lm = loss()
            fac_v[n][i + p.dims[n] * j] = old
            assert abs((lp - lm) / (2 * h) - dU[0][n][i, j]) <= 1e-5 * scale


def test_backward_mixed_autograd_function(cuda_lib):
    from paper_2603_13532_gb300 import binding
    probs = _mixed_problems(1)
    plan = binding.Plan(probs, kind="krp", precision="mixed", seed=5)
    Qs, Ts = _qs_and_targets(plan, probs, 5)
    Q = plan.pack_bases(Qs)
    T = plan.pack_core(Ts)
    x = plan.flat_inputs
    x.requires_grad_(True)
    H = binding.ProjectCore.apply(x, Q, plan)
    L = ((H - T) ** 2).sum()
    (gx,) = torch.autograd.grad(L, [x])
    x.requires_grad_(False)
    direct = plan.backward(Qs, [2.0 * (h - t) for h, t in zip(plan.project(Qs), Ts)])
    # the autograd gradient lands in the inputs' dtype (bfloat16): compare at bf16 resolution
    g = gx.detach().to(torch.float64).cpu().numpy()
    base = x.storage_offset()
    for p, (core_v, fac_v), (dG, dU) in zip(probs, plan.inputs, direct):
        o = core_v.storage_offset() - base
        flat_dG = np.concatenate([a.ravel(order="F") for a in dG])
        assert np.allclose(g[o: o + flat_dG.size], flat_dG, rtol=1e-2, atol=1e-2 * np.abs(flat_dG).max())

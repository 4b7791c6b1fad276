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


def test_backward_rejects_mixed_plans(cuda_lib):
    from paper_2603_13532_gb300 import binding
    g = np.random.default_rng(9)
    dims = [16, 24, 32]
    prob = wl._finish([wl.Problem(dims, [g.standard_normal((2, 2, 2))],
                                  [[g.standard_normal((n, 2)) for n in dims]], [3, 3, 3], [1, 1, 1])], True)
    plan = binding.Plan(prob, kind="krp", precision="mixed", seed=1)
    Q = torch.zeros(plan.info.basis_elems, dtype=torch.float64, device="cuda")
    Hb = torch.zeros(plan.info.core_elems, dtype=torch.float64, device="cuda")
    dc = torch.zeros(max(1, plan.info.grad_core_elems), dtype=torch.float64, device="cuda")
    df = torch.zeros(max(1, plan.info.grad_factor_elems), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.TksError) as e:
        plan.backward_raw(Q, Hb, dc, df)
    assert e.value.code == 7

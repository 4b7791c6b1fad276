"""tucker_sum_sketch_noalloc: the structured sketch for callers that cannot allocate device memory.

It must give what tucker_sum_sketch gives (FP64, the same problem alone in a plan) while using
only its static device scratch; two calls in a row with different problems (synchronized between
the calls, and enqueued back to back on one stream) check that the reused scratch carries nothing
over from one call to the next.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problem_t(binding, prob, views, keep):
    core_t, facs = views
    d = prob.order
    dims = (ctypes.c_int64 * d)(*prob.dims)
    ranks = (ctypes.c_int32 * (prob.num_terms * d))(*[r for rk in prob.ranks() for r in rk])
    tgt = (ctypes.c_int32 * d)(*prob.target)
    ovs = (ctypes.c_int32 * d)(*prob.oversampling)
    fptrs = (ctypes.c_void_p * d)(*[f.data_ptr() for f in facs])
    alpha = (ctypes.c_double * prob.num_terms)(*prob.alpha) if prob.alpha is not None else None
    keep += [dims, ranks, tgt, ovs, fptrs, alpha]
    return binding.Problem_t(d, dims, prob.num_terms, ranks, tgt, ovs,
                             ctypes.cast(alpha, ctypes.POINTER(ctypes.c_double)) if alpha else None,
                             ctypes.c_void_p(core_t.data_ptr()), fptrs)


def _reference_sketch(binding, prob, kind, seed, omega_lowprec=False):
    plan = binding.Plan([prob], kind=kind, precision="fp64", seed=seed, omega_lowprec=omega_lowprec)
    return plan.sketch()[0], plan.pinfo[0]


def _problems(seed):
    g = np.random.default_rng(seed)
    probs = []
    for dims, K in ([[70, 33, 41], 4], [[17, 65, 23], 3]):
        cores, facs = [], []
        for _ in range(K):
            r = [int(x) for x in g.integers(1, 7, size=3)]
            cores.append(g.standard_normal(r))
            facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
        probs.append(wl.Problem(dims, cores, facs, [5, 6, 4], [2, 1, 3], alpha=list(g.standard_normal(K))))
    return probs


def _unpack(Y, prob, pinfo):
    host = Y.cpu().numpy()
    out, off = [], 0
    for m in range(prob.order):
        S = pinfo.sketch_cols[m]
        out.append(host[off: off + prob.dims[m] * S].reshape(prob.dims[m], S, order="F"))
        off += prob.dims[m] * S
    return out


def _assert_close(got, ref, what):
    for m, (a, b) in enumerate(zip(got, ref)):
        err = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert err <= 1e-12, (what, m, err)


@pytest.mark.parametrize("kind", ["krp", "kron"])
@pytest.mark.parametrize("omega_lowprec", [0, 1])
def test_noalloc_sketch_matches_tucker_sum_sketch_twice(cuda_lib, kind, omega_lowprec):
    from paper_2603_13532_gb300 import binding
    lib = binding.load()
    probs = _problems(42)
    seed = 77
    prm = binding.Params_t(binding.SKETCH[kind], 0, 0, seed, 0.0, omega_lowprec, 0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for prob in probs:                      # two calls in a row, different problems
        ref, pinfo = _reference_sketch(binding, prob, kind, seed, bool(omega_lowprec))
        flat, views = binding.pack_inputs([prob], "fp64", torch.device("cuda"))
        keep = []
        pt = _problem_t(binding, prob, views[0], keep)
        total = sum(prob.dims[m] * pinfo.sketch_cols[m] for m in range(3))
        Y = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.tucker_sum_sketch_noalloc(ctypes.byref(pt), ctypes.byref(prm), ctypes.c_void_p(Y.data_ptr()),
                                           stream)
        assert rc == 0, lib.tks_last_error()
        torch.cuda.synchronize()
        _assert_close(_unpack(Y, prob, pinfo), ref, (kind, omega_lowprec))


@pytest.mark.parametrize("kind", ["krp", "kron"])
def test_noalloc_two_calls_back_to_back_on_one_stream(cuda_lib, kind):
    """Both problems enqueued on one stream with no synchronization between them: the second
    call's table copy is ordered after the first call's kernels, so both results stand."""
    from paper_2603_13532_gb300 import binding
    lib = binding.load()
    probs = _problems(43)
    seed = 78
    prm = binding.Params_t(binding.SKETCH[kind], 0, 0, seed, 0.0, 0, 0)
    refs = [_reference_sketch(binding, prob, kind, seed) for prob in probs]
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    keep, outs = [], []
    for prob, (_, pinfo) in zip(probs, refs):
        flat, views = binding.pack_inputs([prob], "fp64", torch.device("cuda"))
        pt = _problem_t(binding, prob, views[0], keep)
        keep += [flat, pt]
        total = sum(prob.dims[m] * pinfo.sketch_cols[m] for m in range(3))
        Y = torch.full((total,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.tucker_sum_sketch_noalloc(ctypes.byref(pt), ctypes.byref(prm), ctypes.c_void_p(Y.data_ptr()),
                                           stream)
        assert rc == 0, lib.tks_last_error()
        outs.append(Y)
    torch.cuda.synchronize()
    for prob, (ref, pinfo), Y in zip(probs, refs, outs):
        _assert_close(_unpack(Y, prob, pinfo), ref, kind)


def test_noalloc_rejects_problems_beyond_the_static_scratch(cuda_lib):
    from paper_2603_13532_gb300 import binding
    lib = binding.load()
    d = 3
    dims = (ctypes.c_int64 * d)(4096, 4096, 4096)
    K = 64
    ranks = (ctypes.c_int32 * (K * d))(*([32] * (K * d)))
    tgt = (ctypes.c_int32 * d)(60, 60, 60)
    ovs = (ctypes.c_int32 * d)(4, 4, 4)
    facs = (ctypes.c_void_p * d)(0x1000, 0x1000, 0x1000)
    pt = binding.Problem_t(d, dims, K, ranks, tgt, ovs, None, ctypes.c_void_p(0x1000), facs)
    prm = binding.Params_t(1, 0, 0, 1, 0.0, 0, 0)
    rc = lib.tucker_sum_sketch_noalloc(ctypes.byref(pt), ctypes.byref(prm), ctypes.c_void_p(0x1000), None)
    assert rc == 1
    assert b"static scratch" in lib.tks_last_error()

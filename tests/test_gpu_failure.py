"""Failure paths that can be exercised without faulting the GPU.

* A bounded device-side wait that runs out: the plan's tensor-core GEMMs are told to wait first for a
  device word that nothing sets (tks_plan_set_fault_test), with a short wait bound.  Each kernel then
  takes its timeout exit (records TKS_ETIMEOUT, drains its own copies and products, frees its tensor
  memory, returns), tks_sync_status reports TKS_ETIMEOUT, and the same plan and a fresh one still
  compute correct sketches afterwards.
* A NaN in one core entry: the QR of the sketch sees a non-finite column norm and the call reports
  TKS_ENONFINITE; a fresh plan on clean inputs is unaffected.
"""
import numpy as np
import pytest

from oracle import sketch_sum as ss
from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TIMEOUT, NONFINITE = 4, 5


def _mixed_problems(seed=3):
    g = np.random.default_rng(seed)
    dims = [48, 40, 56]
    cores, facs = [], []
    for _ in range(3):
        r = [int(x) for x in g.integers(3, 8, size=3)]
        cores.append(g.standard_normal(r))
        facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
    return wl._finish([wl.Problem(dims, cores, facs, [8, 8, 8], [3, 3, 3])], True)


def _sketch_err(plan, prob):
    Ys = plan.sketch()[0]
    ref = ss.recompress(prob.terms(), "krp", prob.target, prob.oversampling, seed=plan.seed, rounding="bf16")
    return max(np.linalg.norm(Ys[m] - ref["Y"][m]) / np.linalg.norm(ref["Y"][m]) for m in range(3))


def test_wait_timeout_is_reported_and_the_plan_recovers(cuda_lib):
    from paper_2603_13532_gb300 import binding
    probs = _mixed_problems()
    plan = binding.Plan(probs, kind="krp", precision="mixed", seed=12)
    plan.set_fault_test(wait_cycles=2_000_000, stall=True)     # about 1 ms per wait
    with pytest.raises(binding.TksError) as e:
        plan.sketch()
    assert e.value.code == TIMEOUT
    plan.set_fault_test(wait_cycles=0, stall=False)
    assert _sketch_err(plan, probs[0]) <= 1e-5
    fresh = binding.Plan(probs, kind="krp", precision="mixed", seed=12)
    assert _sketch_err(fresh, probs[0]) <= 1e-5


def test_fault_test_arguments_are_checked(cuda_lib):
    from paper_2603_13532_gb300 import binding
    plan = binding.Plan(_mixed_problems(), kind="krp", precision="mixed", seed=1)
    with pytest.raises(binding.TksError):
        plan.set_fault_test(wait_cycles=-1)
    assert plan.lib.tks_plan_set_fault_test(plan.handle, 0, 2) == 1     # TKS_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nan_core_entry_reports_enonfinite(cuda_lib, precision):
    from paper_2603_13532_gb300 import binding
    w = wl.exact_recovery(n=40, K=3, r=5, target=15)
    probs = w.problems if precision == "fp64" else wl._finish(list(w.problems), True)
    plan = binding.Plan(probs, kind="krp", precision=precision, seed=2)
    plan.inputs[0][0][7] = float("nan")           # one entry of the first core, in place on the device
    with pytest.raises(binding.TksError) as e:
        plan.recompress()
    assert e.value.code == NONFINITE
    clean = binding.Plan(probs, kind="krp", precision=precision, seed=2)
    got = clean.recompress()[0]
    assert all(np.isfinite(got["core"]).ravel())

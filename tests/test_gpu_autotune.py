"""The schedule knobs and the autotuner of tks_plan_create (tks_params.autotune, tks_plan_tuning).

The knobs choose how a result is computed (lanes of concurrent launch sequences, CholeskyQR3 or
Householder for the float64 factorizations, the projection's chunk, the tensor-core ring depth),
never what: every schedule must meet the mixed path's accuracy against the FP64 oracle, and a plan
created from the JSON picks of an autotuned plan must run the same schedule (bit-identical results).
"""
import numpy as np
import pytest

from oracle import sketch_sum as ss
from oracle.tensor import tucker_entries, tucker_full
from paper_2603_13532_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _problems():
    g = np.random.default_rng(77)
    probs = []
    for dims, K in ([[72, 40, 136], 3], [[24, 96, 56], 2], [[64, 64, 64], 4], [[128, 48, 32], 2]):
        cores, facs = [], []
        for _ in range(K):
            r = [int(x) for x in g.integers(2, 9, size=3)]
            cores.append(g.standard_normal(r))
            facs.append([g.standard_normal((n, ri)) for n, ri in zip(dims, r)])
        probs.append(wl.Problem(dims, cores, facs, [6, 7, 5], [2, 3, 2], alpha=list(g.standard_normal(K))))
    return wl._finish(probs, True)


def _check_against_oracle(probs, outs, seed):
    for i, (prob, got) in enumerate(zip(probs, outs)):
        ref = ss.recompress(prob.terms(), "krp", prob.target, prob.oversampling, seed=seed, problem=i,
                            alpha=prob.alpha, rounding="bf16")
        X = sum(a * tucker_full(G, Us) for a, (G, Us) in zip(prob.alpha, prob.terms()))
        Xg = tucker_full(got["core"], got["factors"])
        Xo = tucker_full(ref["core"], ref["factors"])
        nx = np.linalg.norm(X)
        assert np.linalg.norm(Xg - Xo) / nx <= 1e-5
        assert got["ranks"] == ref["ranks"]


@pytest.mark.parametrize("schedule", [{"sketch_qr": 2}, {"hosvd_r": 2}, {"sketch_qr": 3, "hosvd_r": 3},
                                      {"proj_chunk": 8}, {"tc_stages": 2},
                                      {"lanes": 3, "sketch_qr": 2, "hosvd_r": 2, "proj_chunk": 8, "tc_stages": 3}])
def test_every_schedule_meets_the_oracle(cuda_lib, schedule):
    from paper_2603_13532_gb300 import binding
    probs = _problems()
    plan = binding.Plan(probs, kind="krp", precision="mixed", seed=11, schedule=schedule)
    t = plan.tuning()
    assert t["autotuned"] == 0
    for k, v in schedule.items():
        assert t["picked"][k] == v
    _check_against_oracle(probs, plan.recompress(), 11)


def test_autotuned_plan_reports_and_replays_its_schedule(cuda_lib):
    from paper_2603_13532_gb300 import binding
    probs = _problems()
    tuned = binding.Plan(probs, kind="krp", precision="mixed", seed=13, autotune=True)
    t = tuned.tuning()
    assert t["autotuned"] == 1
    assert len(t["candidates"]) >= 6
    assert all(c["ms"] > 0 for c in t["candidates"])
    assert 0 < t["picked_ms"] <= t["rule_ms"]
    assert set(t["picked"]) == set(binding.SCHEDULE_KNOBS)
    out_t = tuned.recompress()
    _check_against_oracle(probs, out_t, 13)
    # the same knobs without autotuning run the same launch sequence: identical results
    again = binding.Plan(probs, kind="krp", precision="mixed", seed=13, schedule=t["picked"])
    for a, b in zip(out_t, again.recompress()):
        assert np.array_equal(a["core"], b["core"])
        for fa, fb in zip(a["factors"], b["factors"]):
            assert np.array_equal(fa, fb)


@pytest.mark.parametrize("schedule", [{"proj_chunk": 5}, {"tc_stages": 1}, {"sketch_qr": 4}, {"hosvd_r": -1},
                                      {"lanes": 9}])
def test_bad_knobs_are_rejected(cuda_lib, schedule):
    from paper_2603_13532_gb300 import binding
    with pytest.raises(binding.TksError) as e:
        binding.Plan(_problems()[:1], kind="krp", precision="mixed", seed=1, schedule=schedule)
    assert e.value.code == 1


@pytest.mark.parametrize("schedule", [{"sketch_qr": 3, "hosvd_r": 3}, {"sketch_qr": 2, "hosvd_r": 2}])
def test_decay512_schedules_meet_the_oracle(cuda_lib, schedule):
    """The ill-conditioned workload (mode spectra decaying like 10^(-i/8): unfoldings with condition
    numbers near 1e7): two-pass CholeskyQR, or Householder throughout, still matches the oracle."""
    from paper_2603_13532_gb300 import binding
    w = wl.decay512()
    p = w.problems[0]
    plan = binding.Plan(w.problems, kind="krp", precision="mixed", seed=w.seed, schedule=schedule)
    ref = ss.recompress(p.terms(), "krp", p.target, p.oversampling, seed=w.seed, problem=0, alpha=p.alpha,
                        rounding="bf16")
    got = plan.recompress()[0]
    assert got["ranks"] == ref["ranks"] == [48, 48, 48]
    idx = np.random.default_rng(1).integers(0, 512, size=(400, 3))
    eg = tucker_entries(got["core"], got["factors"], idx)
    eo = tucker_entries(ref["core"], ref["factors"], idx)
    ex = sum(tucker_entries(G, Us, idx) for G, Us in p.terms())
    scale = np.sqrt(np.mean(ex ** 2))
    assert np.sqrt(np.mean((eg - eo) ** 2)) <= 1e-5 * scale

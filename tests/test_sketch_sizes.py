"""The library's sketch sizes (stage a0: Sec. 3.2 for Khatri-Rao, Eq. heuristic_formula in exact
integer form for Kronecker) through the host-only tks_sketch_sizes, bit for bit against the oracle
and the stored worked values, with the argument checks.  No GPU: the call touches no device."""
import ctypes
import itertools
import json
import math
import os
import random

import pytest

from oracle import sketch_sum as ss

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EINVAL, EUNSUPPORTED = 1, 7


@pytest.fixture(scope="module")
def binding():
    from paper_2603_13532_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def lib_sizes(binding, kind, ell):
    """Sizes for targets ell and no oversampling, or the status code of a refusal."""
    try:
        cols, S = binding.sketch_sizes(kind, list(ell), [0] * len(ell))
    except binding.TksError as e:
        return e.code
    return [cols, S]


def expected(kind, ell):
    cols, S = ss.sketch_sizes(kind, list(ell))
    if kind == "kron" and max(S) > 8192:
        return EUNSUPPORTED
    return [list(cols), list(S)]


def test_worked_values(binding):
    """The stored cases (the configurations' sizes and the exact-root cases, written from the oracle
    and pinned there to Sec. 3.2 and Eq. sketch_condition)."""
    cases = json.load(open(os.path.join(ROOT, "tests", "golden", "sketch_sizes.json")))["cases"]
    for c in cases:
        cols, S = binding.sketch_sizes(c["kind"], c["ell"], [0] * len(c["ell"]))
        assert (cols, S) == (c["cols"], c["S"]), c["name"]


def test_target_plus_oversampling_is_ell(binding):
    """ell_n = target_n + oversampling_n: the split between the two does not matter."""
    assert binding.sketch_sizes("kron", [30, 30, 30], [2, 2, 2]) == binding.sketch_sizes("kron", [32] * 3, [0] * 3)
    assert binding.sketch_sizes("krp", [48, 40, 7], [10, 0, 3]) == ([58] * 3, [58] * 3)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6])
def test_random_ells_match_the_oracle(binding, d):
    rnd = random.Random(1000 + d)
    hi = {2: 4000, 3: 300, 4: 60, 5: 30, 6: 20}[d]
    for _ in range(150):
        ell = [rnd.randint(1, hi) for _ in range(d)]
        for kind in ("krp", "kron"):
            assert lib_sizes(binding, kind, ell) == expected(kind, ell), (kind, ell)


def test_exact_roots(binding):
    """prod_j ell_j a perfect (d-1)-th power times ell_i, where a floating point root can land just
    above an integer: the least s meets (s ell_i)^(d-1) >= prod_j ell_j with equality."""
    for d, base in itertools.product([3, 4, 5], [2, 3, 5, 6, 7, 10, 12]):
        ell = [base] * d
        got = lib_sizes(binding, "kron", ell)
        want = expected("kron", ell)
        assert got == want, ell
        if isinstance(got, list):
            s = got[0][0]
            assert (s * base) ** (d - 1) >= base ** d > ((s - 1) * base) ** (d - 1)


def test_large_ells_stay_exact(binding):
    """Values near the 2^21 limit, with one small mode so that the sketch stays within 8192 columns:
    the integer bisection gives the oracle's exact sizes."""
    cases = [[2 ** 21, 2 ** 21, 1], [8191, 8192, 1], [2 ** 20 + 1, 2 ** 20 - 1, 3], [4096, 4096, 1, 1],
             [2 ** 21, 1, 1, 1, 1, 1], [3 ** 13, 3 ** 13, 1]]
    for ell in cases:
        for kind in ("krp", "kron"):
            assert lib_sizes(binding, kind, ell) == expected(kind, ell), (kind, ell)


def test_sizes_satisfy_the_sketch_condition(binding):
    """Eq. sketch_condition: every Kronecker S_n reaches ell_n and is the product of the other modes'
    s_j."""
    rnd = random.Random(7)
    for _ in range(200):
        d = rnd.randint(2, 6)
        ell = [rnd.randint(1, 24) for _ in range(d)]
        got = lib_sizes(binding, "kron", ell)
        if isinstance(got, list):
            cols, S = got
            assert all(S[n] >= ell[n] for n in range(d))
            assert all(S[n] == math.prod(cols[j] for j in range(d) if j != n) for n in range(d))


def test_rejections(binding):
    lib = binding.load()
    i32 = ctypes.c_int32
    out1, out2 = (i32 * 6)(), (i32 * 6)()

    def call(sketch, order, target, over, a=out1, b=out2):
        t = (i32 * max(1, len(target)))(*target) if target is not None else None
        o = (i32 * max(1, len(over)))(*over) if over is not None else None
        return lib.tks_sketch_sizes(sketch, order, t, o, a, b)

    assert call(1, 3, [4, 4, 4], [0, 0, 0]) == 0
    assert call(2, 3, [4, 4, 4], [0, 0, 0]) == EINVAL        # unknown sketch
    assert call(0, 1, [4], [0]) == EINVAL                    # order below 2
    assert call(0, 7, [4] * 7, [0] * 7) == EINVAL            # order above the maximum
    assert call(0, 3, [4, 0, 4], [0, 0, 0]) == EINVAL        # target below 1
    assert call(0, 3, [4, 4, 4], [0, -1, 0]) == EINVAL       # negative oversampling
    assert call(1, 3, [2 ** 21, 4, 4], [1, 0, 0]) == EINVAL  # ell above 2^21
    assert call(1, 3, [2 ** 31 - 1, 4, 4], [2 ** 31 - 1, 0, 0]) == EINVAL   # no int overflow
    assert call(0, 3, None, [0, 0, 0]) == EINVAL
    assert call(0, 3, [4, 4, 4], None) == EINVAL
    assert call(0, 3, [4, 4, 4], [0, 0, 0], a=None) == EINVAL
    assert call(0, 3, [4, 4, 4], [0, 0, 0], b=None) == EINVAL
    assert call(0, 3, [9000, 9000, 9000], [0, 0, 0]) == EUNSUPPORTED   # Kronecker wider than 8192
    assert b"8192" in lib.tks_last_error()

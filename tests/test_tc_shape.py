"""The tensor-core GEMM's launch shape (csrc/tc_shape.h), built for the host.

Every launch must fit the SM: at most 227 KB of dynamic shared memory per CTA, 228 KB per SM with
1 KB reserved per CTA, and 512 TMEM columns.  A CTA allocates acc x 64 columns, so four
accumulators (256 columns) are only safe where exactly two CTAs fit an SM by shared memory, and
eight (512 columns) only where one does; a third CTA, or a second beside eight accumulators, would
wait for columns.  The rule itself: two CTAs per SM when K <= 1024 and either at most 4,864 tiles
or K <= 256 (four k-blocks), unless the launch runs beside other lanes' kernels (allow_two = 0),
which always takes one CTA per SM.  The kernel gives each job four accumulators when its K <= 1024
and eight above, so a two-CTA launch (K <= 1024 throughout) never needs more than it allocates.
"""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_2603_13532_gb300" / "csrc"

SM_SMEM = 228 * 1024          # shared memory of one SM
CTA_RESERVED = 1024           # reserved by the system for each resident CTA
CTA_MAX_DYN = 227 * 1024      # opt-in limit of one CTA's dynamic shared memory
TMEM_COLS = 512


@pytest.fixture(scope="module")
def shapes(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("tc_shape") / "tc_shape_harness"
    subprocess.run([gxx, "-O2", "-std=c++17", f"-I{CSRC}", str(ROOT / "tests" / "tc_shape_harness.cpp"),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    rows = [tuple(int(v) for v in line.split()) for line in out.splitlines()]
    assert len(rows) == 15 * 8 * 3 * 3 * 5 * 2
    return rows


def ctas_per_sm(smem):
    return SM_SMEM // (smem + CTA_RESERVED)


def test_every_shape_fits_the_sm(shapes):
    for km, tiles, na, nb, ms, allow, two, stages, smem, acc, need in shapes:
        case = (km, tiles, na, nb, ms)
        assert 1 <= stages <= 4, case
        assert smem >= need and smem <= CTA_MAX_DYN, case
        assert ms == 0 or stages <= ms, case
        # the TMEM columns of the CTAs that shared memory lets onto one SM never exceed 512
        assert ctas_per_sm(smem) * acc * 64 <= TMEM_COLS, case
        if two:
            assert acc == 4 and ctas_per_sm(smem) == 2, case
        else:
            assert acc == 8 and ctas_per_sm(smem) == 1, case


def test_rule_and_rounding(shapes):
    for km, tiles, na, nb, ms, allow, two, stages, smem, acc, need in shapes:
        expect = bool(allow) and km <= 1024 and (tiles <= 4864 or km <= 256)
        assert bool(two) == expect, (km, tiles)
        nk = -(-km // 64)
        if two:
            # at most four k-blocks per float32 accumulator
            assert -(-nk // acc) <= 4, (km, tiles)
        # the kernel's per-job count: four accumulators up to K = 1024, eight above; a CTA
        # allocates at least that many for every job it can be given
        assert (4 if km <= 1024 else 8) <= acc, (km, tiles, two)


def test_deepest_ring_that_fits(shapes):
    """The ring is the deepest of 4, 3, 2 stages within the CTA's budget (112 KB on two CTAs, 220 KB
    alone), else one stage; the tile sizes are 128 x 64 A planes and 64 x 64 B planes of bf16."""
    def ring_bytes(s, na, nb):
        return 1024 + s * (na * 128 * 64 * 2 + nb * 64 * 64 * 2) + 8 * (2 * s + 1) + 16

    for km, tiles, na, nb, ms, allow, two, stages, smem, acc, need in shapes:
        assert need == ring_bytes(stages, na, nb)
        budget = 112 * 1024 if two else 220 * 1024
        deepest = next((s for s in (4, 3, 2) if ring_bytes(s, na, nb) <= budget), 1)
        assert stages == (min(deepest, ms) if ms > 0 else deepest), (km, tiles, na, nb, ms)


def test_measured_launches(shapes):
    """The decay512 x 152 launches (a2: 1 x 1 planes, K = 512, 760 tiles; a4: 1 x 3, K ~ 640, 608
    tiles; a6: 1 x 3, K = 512, 760 tiles) run two CTAs per SM; the order-4 Kronecker Y = Ucat Vcat
    (K = 896, about 108,000 tiles) and H = Tcat A^T (3 x 3 planes, K = 896, about 19,000 tiles)
    one; the backward's K = 40 launches of 15,200 and 5,472 tiles two."""
    by = {(r[0], r[1], r[2], r[3], r[4], r[5]): r for r in shapes}
    assert by[(512, 760, 1, 1, 0, 1)][6:8] == (1, 4)
    assert by[(640, 760, 1, 3, 0, 1)][6:8] == (1, 2)
    assert by[(896, 108000, 1, 3, 0, 1)][6] == 0
    assert by[(896, 15200, 3, 3, 0, 1)][6] == 0
    assert by[(40, 15200, 3, 3, 0, 1)][6:8] == (1, 1)
    # a lane of a multi-lane plan: one CTA per SM whatever the shape
    assert by[(512, 760, 1, 1, 0, 0)][6] == 0 and by[(40, 15200, 3, 3, 0, 0)][6] == 0

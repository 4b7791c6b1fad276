"""The digit-product kernels' float64 composition (csrc/compose.cuh), built for the host.

N = hi 2^28 + lo is an exact integer (the combined level sums) and the kernels need N 2^scale rounded
once to nearest-even.  Python's Fraction -> float conversion rounds a rational exactly that way, so
each case is checked bit for bit against it: random operands over the ranges the kernels produce,
both signs and cancellation between hi and lo, carries into the next binade, and exact ties.
"""
import random
import shutil
import struct
import subprocess
from fractions import Fraction
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_2603_13532_gb300" / "csrc"


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("compose") / "compose_harness"
    subprocess.run([gxx, "-O2", "-std=c++17", f"-I{CSRC}", str(ROOT / "tests" / "compose_harness.cpp"),
                    "-o", str(exe)], check=True)
    return exe


def exact(hi, lo, scale):
    n = hi * (1 << 28) + lo
    return float(Fraction(n) * (Fraction(2) ** scale)) if n else 0.0


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def cases(rng):
    out = []
    for _ in range(20000):                      # the kernels' ranges: |hi|, |lo| < 2^47
        hi = rng.randrange(-(1 << 47), 1 << 47)
        lo = rng.randrange(-(1 << 47), 1 << 47)
        out.append((hi, lo, rng.randrange(-200, 60)))
    for _ in range(5000):                       # any width up to 2^59, small operands
        bh, bl = rng.randrange(0, 60), rng.randrange(0, 60)
        hi = rng.randrange(-(1 << bh), (1 << bh) + 1)
        lo = rng.randrange(-(1 << bl), (1 << bl) + 1)
        out.append((hi, lo, rng.randrange(-300, 100)))
    for _ in range(3000):                       # cancellation: lo close to -hi 2^28
        hi = rng.randrange(-(1 << 30), 1 << 30)
        lo = -hi * (1 << 28) + rng.randrange(-(1 << 20), 1 << 20)
        if abs(lo) < (1 << 59):
            out.append((hi, lo, rng.randrange(-60, 60)))
    for _ in range(3000):                       # exact ties and the bits around them: N = m 2^k +- d
        k = rng.randrange(1, 22)
        m = rng.randrange(1 << 52, 1 << 53) * 2 + 1       # odd: 54 significant bits, the last a half ulp
        n = (m << k) + rng.choice([0, 0, 1, -1])
        n = -n if rng.random() < 0.5 else n
        hi, lo = n >> 28, n & ((1 << 28) - 1)
        out.append((hi, lo, rng.randrange(-120, 0)))
    for m in (1 << 53) - 1, (1 << 54) - 1, (1 << 53) + 1:  # rounding carries into the next binade
        for sh in (0, 3, 10):
            n = m << sh
            out.append((n >> 28, n & ((1 << 28) - 1), -70))
    out += [(0, 0, 0), (0, 1, -10), (0, -1, 5), (1, 0, 0), (-1, 0, 0), (0, (1 << 28) - 1, 0), (-1, 1, 3)]
    return out


def test_compose_rounds_exactly(harness):
    rng = random.Random(20260315)
    cs = cases(rng)
    inp = "".join(f"{h} {l} {s}\n" for h, l, s in cs)
    res = subprocess.run([str(harness)], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (h, l, s), line in zip(cs, res):
        want = bits(exact(h, l, s))
        a, b = (int(x, 16) for x in line.split())
        assert a == want, (h, l, s, hex(a), hex(want))
        assert b == want, (h, l, s, hex(b), hex(want))

"""The bf16 helpers of the mixed path (csrc/bf16.cuh), built for the host through tests/host_shim.

* f32_to_f64_exact (the float32 -> float64 widening by the bits) equals the IEEE conversion for
  every class of float32 (normal, subnormal, zero, infinity, NaN).
* split3 carries a float32 or float64 value v into three bfloat16 planes with
  |v - (h0 + h1 + h2)| <= 2^-24 |v| (each plane takes the next 8 significant bits; the float64
  path adds the bits below float32 to the first remainder), h0 is v rounded to float32 and then to
  bfloat16 (round-to-nearest-even), and a float64 that is a float32 value splits exactly as that
  float32 does.
"""
import random
import shutil
import struct
import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_2603_13532_gb300" / "csrc"


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("bf16") / "bf16_harness"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", f"-I{ROOT / 'tests' / 'host_shim'}",
                    f"-I{CSRC}", str(ROOT / "tests" / "bf16_harness.cpp"), "-o", str(exe)], check=True)
    return exe


def run(exe, lines):
    out = subprocess.run([str(exe)], input="".join(lines), capture_output=True, text=True, check=True).stdout
    rows = [r.split() for r in out.splitlines()]
    assert len(rows) == len(lines)
    return rows


def bf16_value(h):
    return float(np.uint32(int(h, 16) << 16).view(np.float32))


def rne_bf16_of_f32(x):
    """bfloat16 pattern of the float32 x, round to nearest, ties to even (the format's definition)."""
    b = int(np.float32(x).view(np.uint32))
    return (b + 0x7FFF + ((b >> 16) & 1)) >> 16


def d_bits(v):
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def f_bits(v):
    return struct.unpack("<I", struct.pack("<f", v))[0]


def test_f32_to_f64_exact_every_class(harness):
    rnd = random.Random(3)
    pats = [0, 0x80000000, 1, 0x807FFFFF, 0x00800000, 0x7F7FFFFF, 0xFF7FFFFF, 0x7F800000, 0xFF800000,
            0x7FC00000, 0x3F800000, 0xBF800001]
    pats += [rnd.getrandbits(32) for _ in range(3000)]
    rows = run(harness, [f"f {p:08x}\n" for p in pats])
    for p, r in zip(pats, rows):
        got = np.uint64(int(r[3], 16)).view(np.float64)
        want = np.float64(np.uint32(p).view(np.float32))
        if np.isnan(want):
            assert np.isnan(got), hex(p)
        else:
            assert got.view(np.uint64) == want.view(np.uint64), hex(p)


def split_error_ok(v, row):
    h = [bf16_value(x) for x in row[:3]]
    # the planes' sum is exact in float64 (24 significant bits spread over three exponents)
    return abs(v - (h[0] + h[1] + h[2])) <= 2.0 ** -24 * abs(v)


def test_split3_float64(harness):
    rnd = random.Random(5)
    vals = [1.0, -1.0, 1.0 + 2.0 ** -52, 3.0 ** 0.5, -(2.0 ** 100) / 3.0, 2.0 ** -100 * 7.0 / 3.0]
    for _ in range(4000):
        e = rnd.choice([rnd.uniform(-20, 20), rnd.uniform(-100, 120)])
        vals.append(rnd.choice([-1.0, 1.0]) * rnd.uniform(1.0, 2.0) * 2.0 ** int(e))
    # values whose float32 rounding is a tie (the 29 dropped bits are exactly half) and near-ties
    for _ in range(500):
        m = rnd.getrandbits(23) | (1 << 23)
        for low in (0x10000000, 0x0FFFFFFF, 0x10000001):
            vals.append(float((m << 29) | low) * 2.0 ** (rnd.randint(-60, 60) - 52))
    rows = run(harness, [f"d {d_bits(v):016x}\n" for v in vals])
    for v, r in zip(vals, rows):
        assert split_error_ok(v, r), (v, r)
        assert int(r[0], 16) == rne_bf16_of_f32(np.float32(v)), (v, r)


def test_split3_float32_and_agreement(harness):
    rnd = random.Random(9)
    vals = [np.float32(rnd.uniform(1.0, 2.0) * 2.0 ** rnd.randint(-90, 100)) * rnd.choice([-1, 1])
            for _ in range(3000)]
    rows_f = run(harness, [f"f {f_bits(float(v)):08x}\n" for v in vals])
    rows_d = run(harness, [f"d {d_bits(float(v)):016x}\n" for v in vals])
    for v, rf, rd in zip(vals, rows_f, rows_d):
        assert split_error_ok(float(v), rf), (v, rf)
        assert rf[:3] == rd[:3], (v, rf, rd)

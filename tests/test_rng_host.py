"""The device RNG (csrc/rng.cuh, stage a1's Gaussian draws), built for the host, against the
oracle's independent restatement (oracle/rng.py) bit for bit.

Both follow one published definition (Philox4x64-10, Box-Muller, series ln and sincos in correctly
rounded IEEE operations in one fixed order), so any disagreement is a transcription error on one
side.  The host build replaces the device's explicitly rounded intrinsics with plain IEEE
arithmetic without contraction (tests/host_shim); the GPU tests compare the device's own draws
with the oracle.
"""
import random
import shutil
import subprocess
from pathlib import Path

import numpy as np
import pytest

from oracle import rng

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_2603_13532_gb300" / "csrc"


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("rng") / "rng_harness"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", f"-I{ROOT / 'tests' / 'host_shim'}",
                    f"-I{CSRC}", str(ROOT / "tests" / "rng_harness.cpp"), "-o", str(exe)], check=True)
    return exe


def run(exe, cases):
    inp = "".join(f"{s} {p} {m} {st} {b}\n" for s, p, m, st, b in cases)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
    rows = [line.split() for line in out.splitlines()]
    assert len(rows) == len(cases)
    z = np.array([[int(v, 16) for v in r[:4]] for r in rows], dtype=np.uint64).view(np.float64)
    f = np.array([[int(v, 16) for v in r[4:8]] for r in rows], dtype=np.uint32).view(np.float32)
    h = np.array([[int(v, 16) for v in r[8:]] for r in rows], dtype=np.uint32)
    return z, f, h


def cases():
    rnd = random.Random(11)
    out = [(0, 0, 0, 0, 0), (20260315, 0, 0, 0, 0), (20260315, 151, 2, 0, 7423),
           (2 ** 64 - 1, 2 ** 32, 5, 0, 2 ** 40 + 3), (1, 2, 3, 4, 5)]
    for _ in range(300):
        out.append((rnd.getrandbits(64), rnd.randrange(512), rnd.randrange(6), rnd.choice([0, 0, 1]),
                    rnd.getrandbits(rnd.choice([8, 20, 40, 62]))))
    return out


def oracle_block(seed, problem, mode, stream, block):
    idx = np.arange(4, dtype=np.int64) + 4 * block
    z = rng.gaussian(seed, problem, mode, idx, stream=stream)
    f = rng.gaussian_f32(seed, problem, mode, idx, stream=stream)
    return z, f


def test_float64_draws_bit_for_bit(harness):
    cs = [c for c in cases() if c[4] < 2 ** 61]     # index 4 block + lane within int64
    z, _, _ = run(harness, cs)
    for i, c in enumerate(cs):
        want, _ = oracle_block(*c)
        assert np.array_equal(z[i].view(np.uint64), want.view(np.uint64)), c


def test_float32_and_bf16_draws_bit_for_bit(harness):
    cs = [c for c in cases() if c[4] < 2 ** 61]
    _, f, h = run(harness, cs)
    for i, c in enumerate(cs):
        _, want = oracle_block(*c)
        assert np.array_equal(f[i].view(np.uint32), want.view(np.uint32)), c
        bf = rng.round_bf16(want).astype(np.float32).view(np.uint32) >> np.uint32(16)
        assert np.array_equal(h[i], bf), c


def test_omega_matrix_layout(harness):
    """Omega_j's column-major element e is lane e % 4 of block e // 4: a 7 x 5 matrix from the
    harness's blocks equals the oracle's omega()."""
    seed, problem, mode, n, s = 99, 4, 2, 7, 5
    blocks = [(seed, problem, mode, 0, b) for b in range((n * s + 3) // 4)]
    z, _, h = run(harness, blocks)
    flat = z.reshape(-1)[: n * s]
    assert np.array_equal(flat.reshape(n, s, order="F"), rng.omega(seed, problem, mode, n, s))
    bf = (h.reshape(-1)[: n * s].astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    assert np.array_equal(bf.reshape(n, s, order="F"), rng.omega(seed, problem, mode, n, s, rounding="bf16"))

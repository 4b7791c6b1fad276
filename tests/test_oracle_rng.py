"""Pins for the oracle's counter-based Gaussian generator (oracle/rng.py).

The generator is pinned to things outside itself: numpy's independent
Philox4x64-10 bit generator, mpmath's arbitrary-precision ln/cos/sin, the
standard normal law (moments, Kolmogorov-Smirnov), and torch's float->bf16
conversion.
"""
import mpmath
import numpy as np
import pytest
from scipy import stats

from oracle import rng


def _numpy_philox_blocks(key, counter, nblocks):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(counter, dtype=np.uint64))
    return bg.random_raw(4 * nblocks).reshape(nblocks, 4)


@pytest.mark.parametrize("key,counter", [
    ((0, 0), (0, 0, 0, 0)),
    ((20260315, 0), (0, 2, 7, 0)),
    ((2**64 - 1, 0), (2**40 + 3, 1, 255, 9)),
])
def test_philox_matches_numpy(key, counter):
    # numpy increments the 256-bit counter before each block; block i is counter + i + 1
    nb = 16
    ref = _numpy_philox_blocks(key, counter, nb)
    c0 = np.arange(counter[0] + 1, counter[0] + 1 + nb, dtype=np.uint64)
    out = rng.philox4x64_10(c0, counter[1], counter[2], counter[3], key[0], key[1])
    np.testing.assert_array_equal(np.stack(out, axis=1), ref)


def test_uniform_open_interval_exact():
    w = np.array([0, 1, 2**12 - 1, 2**12, 2**63, 2**64 - 1], dtype=np.uint64)
    u = rng.uniform_open01(w)
    assert u[0] == 2.0 ** -53 and u[2] == 2.0 ** -53
    assert u[3] == 1.5 * 2.0 ** -52
    assert u[-1] == 1.0 - 2.0 ** -53
    assert np.all((u > 0) & (u < 1))


def _ulp_err(x, ref):
    return abs(float(x) - float(ref)) / float(np.spacing(abs(float(ref))))


def test_ln_within_two_ulp():
    # the reduction u = m 2^e with e = -1 and m near sqrt(2) partly cancels e ln2 against
    # ln m; the result stays within 2 ulp of the exact logarithm
    g = np.random.default_rng(1)
    u = np.concatenate([
        rng.uniform_open01(g.integers(0, 2**63, size=400, dtype=np.uint64) * np.uint64(2)),
        [2.0 ** -53, 2.0 ** -52, 0.5, 0.5 + 2**-53, 1 - 2.0 ** -53, 1 - 2.0 ** -20,
         np.sqrt(0.5), np.nextafter(np.sqrt(0.5), 0), np.nextafter(np.sqrt(0.5), 1), 0.75, 1e-10],
    ])
    out = rng.ln(u)
    mpmath.mp.prec = 120
    worst = max(_ulp_err(o, mpmath.log(mpmath.mpf(float(x)))) for o, x in zip(out, u))
    assert worst <= 2.0, worst


def test_sincos_2pi_accuracy():
    g = np.random.default_rng(2)
    u = np.concatenate([g.random(400), [2.0 ** -53, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75,
                                         0.875, 1 - 2.0 ** -53, 1 / 3, 0.9999]])
    c, s = rng.sincos_2pi(u)
    mpmath.mp.prec = 120
    for ci, si, ui in zip(c, s, u):
        ang = 2 * mpmath.pi * mpmath.mpf(float(ui))
        # absolute error against the exact value at the exact argument
        assert abs(float(ci) - float(mpmath.cos(ang))) <= 3e-16
        assert abs(float(si) - float(mpmath.sin(ang))) <= 3e-16


def test_gaussian_lane_layout_is_box_muller():
    # element e is lane e % 4 of Philox block e // 4 (see oracle/rng.py docstring)
    seed, prob, mode = 77, 3, 1
    idx = np.arange(16)
    z = rng.gaussian(seed, prob, mode, idx)
    w = rng.philox4x64_10(np.arange(4, dtype=np.uint64), mode, prob, 0, seed, 0)
    u = [rng.uniform_open01(x) for x in w]
    mpmath.mp.prec = 120
    for e in idx:
        b, lane = e // 4, e % 4
        u1, u2 = (u[0][b], u[1][b]) if lane < 2 else (u[2][b], u[3][b])
        r = mpmath.sqrt(-2 * mpmath.log(mpmath.mpf(float(u1))))
        ang = 2 * mpmath.pi * mpmath.mpf(float(u2))
        ref = r * (mpmath.cos(ang) if lane % 2 == 0 else mpmath.sin(ang))
        assert abs(float(z[e]) - float(ref)) <= 4e-15 * max(1.0, abs(float(ref)))


def test_gaussian_statistics():
    n = 1_000_000
    z = rng.gaussian(20260315, 0, 0, np.arange(n))
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # different modes / problems are different streams
    z2 = rng.gaussian(20260315, 0, 1, np.arange(n))
    z3 = rng.gaussian(20260315, 1, 0, np.arange(n))
    assert abs(np.corrcoef(z, z2)[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(z, z3)[0, 1]) < 5 / np.sqrt(n)
    # lanes within a block are uncorrelated (Box-Muller cos/sin pair)
    assert abs(np.corrcoef(z[0::4], z[1::4])[0, 1]) < 5 / np.sqrt(n / 4)


def test_omega_column_major_and_bf16_rounding():
    import torch
    Om = rng.omega(5, 2, 1, 7, 3)
    flat = rng.gaussian(5, 2, 1, np.arange(21))
    np.testing.assert_array_equal(Om[:, 1], flat[7:14])
    ref = torch.from_numpy(Om).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(rng.round_fp32_then_bf16(Om), ref)
    # halfway cases round to even
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8)])
    np.testing.assert_array_equal(rng.round_fp32_then_bf16(x), [1.0, 1 + 4 * 2.0 ** -8, -1.0])


# ---- float32 variant used by the low-precision sketch ----------------------

def test_uniform_f32_open_interval_exact():
    w = np.array([0, 2**41 - 1, 2**41, 2**63, 2**64 - 1], dtype=np.uint64)
    u = rng.uniform_open01_f32(w)
    assert u.dtype == np.float32
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24
    assert u[2] == 1.5 * 2.0 ** -23
    assert u[3] == 0.5 + 2.0 ** -24
    assert u[-1] == 1.0 - 2.0 ** -24
    # every value is (j + 1/2) 2^-23 exactly
    j = (w >> np.uint64(41)).astype(np.float64)
    np.testing.assert_array_equal(u.astype(np.float64), (j + 0.5) * 2.0 ** -23)


def _ulp32_err(x, ref):
    return abs(float(x) - float(ref)) / float(np.spacing(np.float32(abs(float(ref)))))


def test_ln_f32_within_two_ulp():
    g = np.random.default_rng(11)
    w = g.integers(0, 2**63, size=3000, dtype=np.uint64) * np.uint64(2)
    u = np.concatenate([rng.uniform_open01_f32(w),
                        np.array([2.0 ** -24, 1.5 * 2.0 ** -23, 0.5, 0.5 + 2.0 ** -24, 1 - 2.0 ** -24,
                                  np.sqrt(0.5), 0.75], dtype=np.float32)]).astype(np.float32)
    out = rng.ln_f32(u)
    assert out.dtype == np.float32
    mpmath.mp.prec = 80
    worst = max(_ulp32_err(o, mpmath.log(mpmath.mpf(float(x)))) for o, x in zip(out, u))
    assert worst <= 2.0, worst


def test_sincos_2pi_f32_accuracy():
    g = np.random.default_rng(12)
    u = np.concatenate([rng.uniform_open01_f32(g.integers(0, 2**63, size=2000, dtype=np.uint64)),
                        np.array([0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 2.0 ** -24,
                                  1 - 2.0 ** -24], dtype=np.float32)]).astype(np.float32)
    c, s = rng.sincos_2pi_f32(u)
    mpmath.mp.prec = 80
    for ci, si, ui in zip(c, s, u):
        ang = 2 * mpmath.pi * mpmath.mpf(float(ui))
        # absolute error at the exact float32 argument, within 1.5 float32 ulp of 1
        assert abs(float(ci) - float(mpmath.cos(ang))) <= 1.8e-7
        assert abs(float(si) - float(mpmath.sin(ang))) <= 1.8e-7


def test_gaussian_f32_lane_layout_is_box_muller():
    seed, prob, mode = 77, 3, 1
    idx = np.arange(16)
    z = rng.gaussian_f32(seed, prob, mode, idx)
    assert z.dtype == np.float32
    w = rng.philox4x64_10(np.arange(4, dtype=np.uint64), mode, prob, 0, seed, 0)
    u = [rng.uniform_open01_f32(x) for x in w]
    mpmath.mp.prec = 80
    for e in idx:
        b, lane = e // 4, e % 4
        u1, u2 = (u[0][b], u[1][b]) if lane < 2 else (u[2][b], u[3][b])
        r = mpmath.sqrt(-2 * mpmath.log(mpmath.mpf(float(u1))))
        ang = 2 * mpmath.pi * mpmath.mpf(float(u2))
        ref = r * (mpmath.cos(ang) if lane % 2 == 0 else mpmath.sin(ang))
        assert abs(float(z[e]) - float(ref)) <= 1e-6 * max(1.0, abs(float(ref)))


def test_gaussian_f32_statistics_and_agreement_with_f64_draws():
    n = 1_000_000
    z = rng.gaussian_f32(20260315, 0, 0, np.arange(n)).astype(np.float64)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # u keeps 23 of the 52 bits of the float64 variant: the two draws agree to ~1e-7
    # except where ln u1 is steep (u1 near 0), and never by more than the 2^-24 shift in u1
    z64 = rng.gaussian(20260315, 0, 0, np.arange(n))
    d = np.abs(z - z64)
    assert np.median(d) < 5e-7
    assert np.mean(d > 1e-4) < 1e-3
    assert d.max() < 0.05


def test_omega_bf16_is_rounded_f32_draws():
    import torch
    Ob = rng.omega(5, 2, 1, 7, 3, rounding="bf16")
    z = rng.gaussian_f32(5, 2, 1, np.arange(21))
    ref = torch.from_numpy(z).to(torch.bfloat16).to(torch.float64).numpy().reshape(7, 3, order="F")
    np.testing.assert_array_equal(Ob, ref)
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8)], dtype=np.float32)
    np.testing.assert_array_equal(rng.round_bf16(x), [1.0, 1 + 4 * 2.0 ** -8, -1.0])

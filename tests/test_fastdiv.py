"""The float32 quotient used by the staging loops of the sketch and projection kernels.

floor(e / d) is taken as trunc((e + 1/2) * RN(1/d)) in float32 (round-to-nearest reciprocal and
product, as the kernels' __frcp_rn and float multiply do); numpy's float32 arithmetic is the same
IEEE arithmetic, so this exhaustive check over the kernels' range is a proof for the device code.
"""
import numpy as np


def _check(emax, dmax):
    e = np.arange(0, emax, dtype=np.int64)
    ef = e.astype(np.float32) + np.float32(0.5)
    for d in range(1, dmax + 1):
        rd = np.float32(1) / np.float32(d)
        q = np.trunc(ef * rd).astype(np.int64)
        assert np.array_equal(q, e // d), d


def test_small_quotient_exact_over_kernel_range():
    _check(1 << 16, 256)
    _check(1 << 15, 1024)

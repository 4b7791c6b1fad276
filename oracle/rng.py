"""Counter-based Gaussian test matrices Omega_j for the sketches (oracle side).

TEST INFRASTRUCTURE ONLY: see ``oracle/__init__.py``.

The paper asks for "standard Gaussian random matrices" Omega_j of size n_j x s
(Khatri-Rao sketch, Sec. 3.1.1, Eq. KRP_sketch) or n_j x s_j (Kronecker sketch,
Sec. 3.1.2), one per mode and reused by the sketches of every other mode
(factor reuse, Sec. 3.1.1).  It does not say how they are drawn.  This module
fixes a definition that a GPU can reproduce bit for bit:

* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): a counter-based bijection of a 4x64-bit counter under a
  2x64-bit key.  Counter = (block, mode, problem, stream), key = (seed, 0).
* Each 64-bit word w becomes u = (floor(w / 2^12) + 1/2) * 2^-52, in (0, 1).
* Box-Muller: z = sqrt(-2 ln u1) * (cos, sin)(2 pi u2).  One Philox block of
  four words gives the four normals of two Box-Muller pairs.
* ln and (cos, sin)(2 pi u) are written here from textbook series -- the
  atanh series ln m = 2 atanh((m-1)/(m+1)) after reduction to [sqrt(1/2),
  sqrt(2)), and the Taylor series of sin and cos on [0, pi/4] after octant
  reduction -- using only operations IEEE 754 rounds correctly (+ - * / sqrt,
  no fused multiply-add), in one fixed order.  numpy's float64 array
  arithmetic obeys exactly that, so any other transcription that performs the
  same operations in the same order gets the same bits.

Element e of Omega (column-major, e = i + n_j * c) is lane e % 4 of block
e // 4.  Lanes 0, 1 are r(w0) cos(2 pi u(w1)), r(w0) sin(2 pi u(w1)); lanes
2, 3 the same for (w2, w3).

The low-precision sketch (``rounding="bf16"``) only needs bfloat16 draws, so it
takes them from a float32 Box-Muller on the same Philox words (``gaussian_f32``):
u = (floor(w / 2^41) + 1/2) * 2^-23 (exact in float32), then the same two series
with float32 coefficients and fewer terms, every step a correctly rounded
float32 operation in one fixed order (numpy's float32 array arithmetic), and the
float32 result rounded to bfloat16 (round-to-nearest-even).
"""
import numpy as np

_U64 = np.uint64
_MASK32 = _U64(0xFFFFFFFF)

# Philox4x64 multipliers and Weyl key increments (Salmon et al. 2011, Table 2).
PHILOX_M0 = _U64(0xD2E7470EE14C6C93)
PHILOX_M1 = _U64(0xCA5A826395121157)
PHILOX_W0 = _U64(0x9E3779B97F4A7C15)
PHILOX_W1 = _U64(0xBB67AE8584CAA73B)
PHILOX_ROUNDS = 10

OMEGA_STREAM = 0  # stream id of the sketch matrices


def _mulhilo64(a, b):
    """Full 128-bit product of uint64 arrays, returned as (high, low) words."""
    a_lo, a_hi = a & _MASK32, a >> _U64(32)
    b_lo, b_hi = b & _MASK32, b >> _U64(32)
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _U64(32)) + (lh & _MASK32) + (hl & _MASK32)
    hi = hh + (lh >> _U64(32)) + (hl >> _U64(32)) + (mid >> _U64(32))
    lo = a * b
    return hi, lo


def philox4x64_10(c0, c1, c2, c3, k0, k1):
    """Philox4x64 with 10 rounds, elementwise over uint64 arrays."""
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.asarray(x, dtype=_U64) for x in (c0, c1, c2, c3))
        k0 = np.asarray(k0, dtype=_U64) + _U64(0)
        k1 = np.asarray(k1, dtype=_U64) + _U64(0)
        for _ in range(PHILOX_ROUNDS):
            hi0, lo0 = _mulhilo64(PHILOX_M0, c0)
            hi1, lo1 = _mulhilo64(PHILOX_M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = k0 + PHILOX_W0
            k1 = k1 + PHILOX_W1
    return c0, c1, c2, c3


def uniform_open01(w):
    """Map uint64 words to doubles in (0, 1): (floor(w/2^12) + 1/2) * 2^-52 (exact)."""
    return ((np.asarray(w, dtype=_U64) >> _U64(12)).astype(np.float64) + 0.5) * 2.0 ** -52


# ---- natural logarithm on (0, 1) ------------------------------------------
_SQRT_HALF = float.fromhex("0x1.6a09e667f3bcdp-1")
_LN2_HI = float.fromhex("0x1.62e42fee00000p-1")   # 32 significant bits: e*_LN2_HI exact
_LN2_LO = float.fromhex("0x1.a39ef35793c76p-33")  # ln 2 - _LN2_HI
# 1/(2k+1), k = 1..11, correctly rounded
_LOG_C = [1.0 / (2 * k + 1) for k in range(1, 12)]


def ln(u):
    """ln u for u in (0, 1) with the atanh series; fixed IEEE operation order.

    u = m 2^e with m in [sqrt(1/2), sqrt(2)); f = (m-1)/(m+1); s = f^2;
    ln m = 2f + (2f s) q(s) with q(s) = sum_{k>=1} s^(k-1)/(2k+1) (Horner,
    11 terms: |f| <= 0.1716 so s^11 < 2^-56); ln u = e ln2_hi + (e ln2_lo + ln m).
    """
    u = np.asarray(u, dtype=np.float64)
    m, e = np.frexp(u)                       # m in [0.5, 1), exact
    low = m < _SQRT_HALF
    m = np.where(low, m * 2.0, m)            # exact
    e = np.where(low, e - 1, e).astype(np.float64)
    f = (m - 1.0) / (m + 1.0)
    s = f * f
    q = np.full_like(s, _LOG_C[-1])
    for c in reversed(_LOG_C[:-1]):
        q = q * s + c
    two_f = f * 2.0
    ln_m = two_f + (two_f * s) * q
    return e * _LN2_HI + (e * _LN2_LO + ln_m)


# ---- (cos, sin)(2 pi u) on (0, 1) -----------------------------------------
_PIO4 = float.fromhex("0x1.921fb54442d18p-1")
_SIN_C = [float.fromhex(h) for h in (
    "-0x1.5555555555555p-3", "0x1.1111111111111p-7", "-0x1.a01a01a01a01ap-13",
    "0x1.71de3a556c734p-19", "-0x1.ae64567f544e4p-26", "0x1.6124613a86d09p-33",
    "-0x1.ae7f3e733b81fp-41", "0x1.952c77030ad4ap-49")]   # (-1)^k/(2k+1)!, k=1..8
_COS_C = [float.fromhex(h) for h in (
    "-0x1.0000000000000p-1", "0x1.5555555555555p-5", "-0x1.6c16c16c16c17p-10",
    "0x1.a01a01a01a01ap-16", "-0x1.27e4fb7789f5cp-22", "0x1.1eed8eff8d898p-29",
    "-0x1.93974a8c07c9dp-37", "0x1.ae7f3e733b81fp-45", "-0x1.6827863b97d97p-53")]  # (-1)^k/(2k)!, k=1..9


def sincos_2pi(u):
    """(cos 2 pi u, sin 2 pi u) for u in (0, 1) by octant reduction + Taylor series.

    x = 8u (exact), k = floor x, f = x - k (exact); the reduced angle is
    t = (pi/4) g with g = f for even k and g = 1 - f (exact) for odd k, so
    that 2 pi u = k pi/4 + (pi/4) f maps onto t in [0, pi/4].
    """
    u = np.asarray(u, dtype=np.float64)
    x = u * 8.0
    k = np.floor(x)
    f = x - k
    k = k.astype(np.int64)
    odd = (k & 1) == 1
    g = np.where(odd, 1.0 - f, f)
    t = g * _PIO4
    s2 = t * t
    p = np.full_like(s2, _SIN_C[-1])
    for c in reversed(_SIN_C[:-1]):
        p = p * s2 + c
    sin_t = t + (t * s2) * p
    q = np.full_like(s2, _COS_C[-1])
    for c in reversed(_COS_C[:-1]):
        q = q * s2 + c
    cos_t = 1.0 + s2 * q
    # octant k: angle k pi/4 + (pi/4) f expressed through t
    swap = (k == 1) | (k == 2) | (k == 5) | (k == 6)
    c_abs = np.where(swap, sin_t, cos_t)
    s_abs = np.where(swap, cos_t, sin_t)
    cos_neg = (k >= 2) & (k <= 5)
    sin_neg = k >= 4
    return np.where(cos_neg, -c_abs, c_abs), np.where(sin_neg, -s_abs, s_abs)


def gaussian(seed, problem, mode, index, stream=OMEGA_STREAM):
    """Standard normal draw number ``index`` (array) of (seed, problem, mode, stream)."""
    index = np.asarray(index, dtype=np.int64)
    block = (index >> 2).astype(_U64)
    lane = index & 3
    w0, w1, w2, w3 = philox4x64_10(block, _U64(mode), _U64(problem), _U64(stream),
                                   _U64(seed), _U64(0))
    first = lane < 2
    u1 = uniform_open01(np.where(first, w0, w2))
    u2 = uniform_open01(np.where(first, w1, w3))
    r = np.sqrt(-2.0 * ln(u1))
    c, s = sincos_2pi(u2)
    return np.where((lane & 1) == 0, r * c, r * s)


# ---- float32 variant (low-precision sketch) -------------------------------
_F32 = np.float32
_SQRT_HALF_F = _F32(float.fromhex("0x1.6a09e6p-1"))
_LN2_HI_F = _F32(float.fromhex("0x1.62e4p-1"))       # 16 significant bits: e*_LN2_HI_F exact
_LN2_LO_F = _F32(float.fromhex("0x1.7f7d1cp-20"))    # ln 2 - _LN2_HI_F, rounded to float32
_LOG_C_F = [_F32(1.0 / (2 * k + 1)) for k in range(1, 6)]   # 1/(2k+1), k = 1..5
_PIO4_F = _F32(float.fromhex("0x1.921fb6p-1"))
_SIN_C_F = [_F32(float.fromhex(h)) for h in (
    "-0x1.555556p-3", "0x1.111112p-7", "-0x1.a01a02p-13", "0x1.71de3ap-19")]          # k = 1..4
_COS_C_F = [_F32(float.fromhex(h)) for h in (
    "-0x1p-1", "0x1.555556p-5", "-0x1.6c16c2p-10", "0x1.a01a02p-16", "-0x1.27e4fcp-22")]  # k = 1..5


def uniform_open01_f32(w):
    """Map uint64 words to float32 in (0, 1): (floor(w/2^41) + 1/2) * 2^-23 (exact)."""
    return ((np.asarray(w, dtype=_U64) >> _U64(41)).astype(_F32) + _F32(0.5)) * _F32(2.0 ** -23)


def ln_f32(u):
    """ln u in float32 for u in (0, 1): the atanh series of ``ln`` with 5 terms.

    |f| <= 0.1716, so the first omitted term s^5/13 is below 2^-27 relative to q.
    Reduction and the split ln 2 = _LN2_HI_F + _LN2_LO_F as in ``ln``; e lies in
    [-23, 0] for the inputs of ``uniform_open01_f32``, so e * _LN2_HI_F is exact.
    """
    u = np.asarray(u, dtype=_F32)
    m, e = np.frexp(u)
    low = m < _SQRT_HALF_F
    m = np.where(low, m * _F32(2.0), m).astype(_F32)
    e = np.where(low, e - 1, e).astype(_F32)
    f = (m - _F32(1.0)) / (m + _F32(1.0))
    s = f * f
    q = np.full_like(s, _LOG_C_F[-1])
    for c in reversed(_LOG_C_F[:-1]):
        q = q * s + c
    two_f = f * _F32(2.0)
    ln_m = two_f + (two_f * s) * q
    return e * _LN2_HI_F + (e * _LN2_LO_F + ln_m)


def sincos_2pi_f32(u):
    """(cos 2 pi u, sin 2 pi u) in float32: the octant reduction of ``sincos_2pi``, then
    Taylor series with 4 (sine) and 5 (cosine) terms; on [0, pi/4] the omitted terms are
    below 2^-28 of the result."""
    u = np.asarray(u, dtype=_F32)
    x = u * _F32(8.0)
    k = np.floor(x)
    f = x - k
    k = k.astype(np.int64)
    odd = (k & 1) == 1
    g = np.where(odd, _F32(1.0) - f, f).astype(_F32)
    t = g * _PIO4_F
    s2 = t * t
    p = np.full_like(s2, _SIN_C_F[-1])
    for c in reversed(_SIN_C_F[:-1]):
        p = p * s2 + c
    sin_t = t + (t * s2) * p
    q = np.full_like(s2, _COS_C_F[-1])
    for c in reversed(_COS_C_F[:-1]):
        q = q * s2 + c
    cos_t = _F32(1.0) + s2 * q
    swap = (k == 1) | (k == 2) | (k == 5) | (k == 6)
    c_abs = np.where(swap, sin_t, cos_t)
    s_abs = np.where(swap, cos_t, sin_t)
    cos_neg = (k >= 2) & (k <= 5)
    sin_neg = k >= 4
    return (np.where(cos_neg, -c_abs, c_abs).astype(_F32),
            np.where(sin_neg, -s_abs, s_abs).astype(_F32))


def gaussian_f32(seed, problem, mode, index, stream=OMEGA_STREAM):
    """float32 standard normal draw ``index`` of (seed, problem, mode, stream): the same
    Philox words and lane layout as ``gaussian``, evaluated in float32."""
    index = np.asarray(index, dtype=np.int64)
    block = (index >> 2).astype(_U64)
    lane = index & 3
    w0, w1, w2, w3 = philox4x64_10(block, _U64(mode), _U64(problem), _U64(stream),
                                   _U64(seed), _U64(0))
    first = lane < 2
    u1 = uniform_open01_f32(np.where(first, w0, w2))
    u2 = uniform_open01_f32(np.where(first, w1, w3))
    r = np.sqrt(_F32(-2.0) * ln_f32(u1))
    c, s = sincos_2pi_f32(u2)
    return np.where((lane & 1) == 0, r * c, r * s).astype(_F32)


def round_bf16(x):
    """float32 -> bfloat16 (round-to-nearest-even), returned as float64 values."""
    b = np.asarray(x, dtype=_F32).view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return (b.astype(np.uint32) << np.uint32(16)).view(_F32).astype(np.float64)


def round_fp32_then_bf16(x):
    """float64 -> float32 (RNE) -> bfloat16 (RNE), returned as float64 values."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return (b.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def omega(seed, problem, mode, n, s, rounding=None):
    """Omega_mode in R^{n x s}, column-major draw order (Sec. 3.1, one per mode)."""
    idx = np.arange(n * s, dtype=np.int64)
    if rounding == "bf16":
        z = round_bf16(gaussian_f32(seed, problem, mode, idx))
    elif rounding is None:
        z = gaussian(seed, problem, mode, idx)
    else:
        raise ValueError(f"unknown rounding {rounding!r}")
    return z.reshape(n, s, order="F")

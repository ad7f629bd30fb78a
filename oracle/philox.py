"""Counter-based Gaussian test matrix for the oracle (Sec. III: "a standard
Gaussian matrix Omega", first step of Algorithms 1 and 3).

TEST INFRASTRUCTURE: only tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.

The paper leaves the random number generator open ("using a random number
generator", Sec. III).  Both sides of this project implement the same
published generator independently, so that Omega is bit-identical on the CPU
and on the GPU:

* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): 10 rounds of the 4x64 S-P network with multipliers
  0xD2E7470EE14C6C93 / 0xCA5A826395121157 and Weyl key increments
  0x9E3779B97F4A7C15 / 0xBB67AE8584CAA73B.
* key = (seed, 0); counter = (g, stream, 0, 0) where g = e // 4 is the group of
  four column-major elements e = i + rows * j of Omega and stream = 0 for Omega.
* each 64-bit word x gives u = ((x >> 41) + 1/2) * 2^-23, a binary32 value
  strictly inside (0, 1) (both steps exact in binary32).
* Box-Muller on the word pairs (w0, w1) -> elements 4g, 4g+1 and
  (w2, w3) -> elements 4g+2, 4g+3: z_even = r cos(2 pi u_b), z_odd = r sin(2 pi u_b),
  r = sqrt(-2 ln u_a).
* the transform runs in IEEE-754 binary32 (the GPU's binary64 rate is a
  small fraction of its binary32 rate), from series written out below using
  only correctly rounded +, -, *, / and sqrt (no fused multiply-add, no
  libm), so every step has exactly one binary32 rounding:
    ln u: u = f 2^e with f in [sqrt(1/2), sqrt(2)); s = (f-1)/(f+1);
          ln f = 2 s (1 + s^2/3 + s^4/5 + ... + s^10/11)  (atanh series;
          |s| <= 0.172, so the next term is below 2^-24 relative);
          ln u = e*ln2 + ln f.
    sin/cos(2 pi u): t = 4u, q = rint(t), r = t - q in [-1/2, 1/2] (exact),
          theta = r * (pi/2); Taylor series of sin and cos to theta^11 and
          theta^12 with coefficients 1/n! rounded to binary32; the quadrant
          q mod 4 selects +-sin / +-cos.
  The binary32 constants (ln 2, pi/2, sqrt(1/2) and the coefficients) are
  the nearest binary32 values of the exact numbers.
* Omega is the binary32 value (exact in binary64 for F64); bf16 / fp16
  round it to the 16-bit format with round-to-nearest-even.
"""
from __future__ import annotations

import math

import numpy as np

_M0 = np.uint64(0xD2E7470EE14C6C93)
_M1 = np.uint64(0xCA5A826395121157)
_W0 = np.uint64(0x9E3779B97F4A7C15)
_W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

_F32 = np.float32
# ln 2, pi/2 and sqrt(1/2) as the nearest binary32 values (0x3F317218,
# 0x3FC90FDB, 0x3F3504F3).
_LN2 = _F32(0.6931471805599453)
_HALF_PI = _F32(1.5707963267948966)
_SQRT_HALF = _F32(0.7071067811865476)

# atanh-series coefficients 1/(2i+1), i = 0..5; sin: (-1)^i / (2i+1)!,
# i = 1..5; cos: (-1)^i / (2i)!, i = 1..6; each the nearest binary32 value
# (the binary64 quotient rounded once more to binary32 lands on it for all
# of these: pinned against exact rationals in the tests).
_LOG_C = [_F32(1.0 / float(2 * i + 1)) for i in range(6)]
_SIN_C = [_F32((-1.0) ** i * (1.0 / float(math.factorial(2 * i + 1)))) for i in range(1, 6)]
_COS_C = [_F32((-1.0) ** i * (1.0 / float(math.factorial(2 * i)))) for i in range(1, 7)]


def _mulhilo(a: np.ndarray, b: np.uint64):
    """64x64 -> 128-bit product, returned as (hi, lo) uint64 arrays."""
    a = a.astype(np.uint64)
    al, ah = a & _LO32, a >> _S32
    bl, bh = b & _LO32, b >> _S32
    with np.errstate(over="ignore"):
        t = al * bl
        u = ah * bl + (t >> _S32)
        v = al * bh + (u & _LO32)
        hi = ah * bh + (u >> _S32) + (v >> _S32)
        lo = a * b
    return hi, lo


def philox4x64_10(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x64 with 10 rounds.  ``ctr``: (N, 4) uint64; ``key``: 2 uint64.

    Returns an (N, 4) uint64 array of output words (SC'11 definition).
    """
    x0, x1, x2, x3 = (ctr[:, i].astype(np.uint64).copy() for i in range(4))
    k0, k1 = np.uint64(key[0]), np.uint64(key[1])
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = np.uint64(k0 + _W0)
                k1 = np.uint64(k1 + _W1)
            hi0, lo0 = _mulhilo(x0, _M0)
            hi1, lo1 = _mulhilo(x2, _M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return np.stack([x0, x1, x2, x3], axis=1)


def uniform_from_u64(x: np.ndarray) -> np.ndarray:
    """Map 64-bit words to binary32 values strictly inside (0, 1) exactly:
    ((x >> 41) + 1/2) * 2^-23 (23-bit integer plus one half: 24 bits)."""
    k = (np.asarray(x, dtype=np.uint64) >> np.uint64(41)).astype(np.float32)
    return (k + _F32(0.5)) * _F32(2.0 ** -23)


def ln_series(u: np.ndarray) -> np.ndarray:
    """Natural log of binary32 u in (0, 1] from the atanh series, every
    operation one binary32 rounding (see module doc)."""
    u = np.asarray(u, dtype=np.float32)
    fr, ex = np.frexp(u)                     # u = fr * 2^ex, fr in [0.5, 1)
    small = fr < _SQRT_HALF
    f = np.where(small, fr * _F32(2.0), fr).astype(np.float32)
    e = np.where(small, ex - 1, ex).astype(np.float32)
    s = (f - _F32(1.0)) / (f + _F32(1.0))
    s2 = s * s
    p = np.full_like(s, _LOG_C[-1])
    for c in reversed(_LOG_C[:-1]):
        p = p * s2
        p = p + c
    lnf = (_F32(2.0) * s) * p
    return e * _LN2 + lnf


def sincos_2pi(u: np.ndarray):
    """(sin(2 pi u), cos(2 pi u)) in binary32 for binary32 u in (0, 1) (see
    module doc)."""
    u = np.asarray(u, dtype=np.float32)
    t = _F32(4.0) * u
    q = np.rint(t)
    r = t - q
    th = r * _HALF_PI
    x2 = th * th
    ps = np.full_like(th, _SIN_C[-1])
    for c in reversed(_SIN_C[:-1]):
        ps = ps * x2
        ps = ps + c
    s = th + (th * x2) * ps
    pc = np.full_like(th, _COS_C[-1])
    for c in reversed(_COS_C[:-1]):
        pc = pc * x2
        pc = pc + c
    c_ = _F32(1.0) + x2 * pc
    quad = q.astype(np.int64) & 3
    sin_v = np.select([quad == 0, quad == 1, quad == 2], [s, c_, -s], -c_)
    cos_v = np.select([quad == 0, quad == 1, quad == 2], [c_, -s, -c_], s)
    return sin_v.astype(np.float32), cos_v.astype(np.float32)


def gaussian_elements(e: np.ndarray, seed: int, stream: int = 0) -> np.ndarray:
    """Standard normal values of the linear element indices ``e`` (binary32
    values, returned as binary64)."""
    e = np.asarray(e, dtype=np.uint64)
    g = e >> np.uint64(2)
    ctr = np.zeros((e.size, 4), dtype=np.uint64)
    ctr[:, 0] = g
    ctr[:, 1] = np.uint64(stream)
    w = philox4x64_10(ctr, (np.uint64(seed & 0xFFFFFFFFFFFFFFFF), np.uint64(0)))
    lane = (e & np.uint64(3)).astype(np.int64)
    hi_pair = lane >= 2
    wa = np.where(hi_pair, w[:, 2], w[:, 0])
    wb = np.where(hi_pair, w[:, 3], w[:, 1])
    ua = uniform_from_u64(wa)
    ub = uniform_from_u64(wb)
    r = np.sqrt(_F32(-2.0) * ln_series(ua))
    sn, cs = sincos_2pi(ub)
    z = np.where((lane & 1) == 0, r * cs, r * sn).astype(np.float32)
    return z.astype(np.float64)             # binary32 values, exact in binary64


def round_fp32(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def round_bf16(x: np.ndarray) -> np.ndarray:
    """binary64 -> fp32 (RNE) -> bf16 (RNE); returned as float64 values."""
    f = round_fp32(x)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    out = (b.astype(np.uint32) << np.uint32(16)).view(np.float32)
    return out.astype(np.float64)


def round_fp16(x: np.ndarray) -> np.ndarray:
    """binary64 -> fp32 (RNE) -> fp16 (RNE); returned as float64 values."""
    return round_fp32(x).astype(np.float16).astype(np.float64)


def round_to(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round binary64 values to the storage precision of ``dtype`` (kept as f64)."""
    if dtype == "f64":
        return np.asarray(x, dtype=np.float64)
    if dtype in ("f32", "tf32"):
        return round_fp32(x).astype(np.float64)
    if dtype == "bf16":
        return round_bf16(x)
    if dtype == "f16":
        return round_fp16(x)
    raise ValueError(f"unknown dtype {dtype!r}")


def gaussian_matrix(rows: int, cols: int, seed: int, stream: int = 0,
                    dtype: str = "f64") -> np.ndarray:
    """Omega (rows x cols), column-major element order, rounded to ``dtype``.

    Returned as a float64 numpy array of shape (rows, cols).
    """
    e = np.arange(rows * cols, dtype=np.uint64)
    z = gaussian_elements(e, seed, stream)
    om = z.reshape(cols, rows).T            # element e = i + rows*j
    return np.ascontiguousarray(round_to(om, dtype))

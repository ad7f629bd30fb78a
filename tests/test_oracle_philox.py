"""Pins of the oracle's Gaussian test matrix (Sec. III, first step of
Algorithms 1 and 3) against things other than itself: the Random123
known-answer vectors, numpy's independent Philox, libm / mpmath, and the
moments and distribution of N(0, 1)."""
import numpy as np
import pytest
from scipy import stats

from conftest import golden_rows
from oracle import philox as ph


def test_philox_known_answer_vectors():
    for row in golden_rows("philox4x64_10_kat.txt"):
        v = [int(x, 16) for x in row]
        ctr = np.array([v[0:4]], dtype=np.uint64)
        out = ph.philox4x64_10(ctr, (np.uint64(v[4]), np.uint64(v[5])))[0]
        assert [int(x) for x in out] == v[6:10]


@pytest.mark.parametrize("seed,stream", [(0, 0), (7, 0), (12345678901234, 3), (2**64 - 1, 1)])
def test_philox_matches_numpy_bitgenerator(seed, stream):
    # numpy increments its 256-bit counter before each block, so a counter
    # one below (c, stream, 0, 0) yields the block for (c, stream, 0, 0).
    for c in (0, 1, 2, 1000, 2**40 + 5):
        start = ((stream << 64) + c - 1) % (1 << 256)
        bg = np.random.Philox(key=seed, counter=start)
        ref = bg.random_raw(4)
        ctr = np.array([[c, stream, 0, 0]], dtype=np.uint64)
        got = ph.philox4x64_10(ctr, (np.uint64(seed), np.uint64(0)))[0]
        assert np.array_equal(ref, got)


def test_uniform_map_exact_and_open_interval():
    x = np.array([0, 1, 2**41 - 1, 2**41, 2**63, 2**64 - 1], dtype=np.uint64)
    u = ph.uniform_from_u64(x)
    assert u.dtype == np.float32
    assert np.all(u > 0) and np.all(u < 1)
    k = u.astype(np.float64) * 2.0**23 - 0.5
    assert np.array_equal(k, np.floor(k))
    assert np.array_equal(k.astype(np.uint64), x >> np.uint64(41))


def test_constants_are_the_nearest_binary32_values():
    # exact rationals (series coefficients) and 120-bit mpmath values
    # (ln 2, pi/2, sqrt(1/2)) rounded once to binary32
    from fractions import Fraction
    import math
    import struct

    def nearest32(q: Fraction) -> float:
        a, e = abs(q), 0
        while Fraction(2) ** e > a:
            e -= 1
        while Fraction(2) ** (e + 1) <= a:
            e += 1
        m = a / Fraction(2) ** (e - 23)
        n, r = divmod(m.numerator, m.denominator)
        rem = Fraction(r, m.denominator)
        if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2):
            n += 1
        v = float(Fraction(n) * Fraction(2) ** (e - 23))
        assert struct.unpack("<f", struct.pack("<f", v))[0] == v
        return -v if q < 0 else v

    assert [float(c) for c in ph._LOG_C] == [nearest32(Fraction(1, 2 * i + 1)) for i in range(6)]
    assert [float(c) for c in ph._SIN_C] == [nearest32(Fraction((-1) ** i, math.factorial(2 * i + 1)))
                                           for i in range(1, 6)]
    assert [float(c) for c in ph._COS_C] == [nearest32(Fraction((-1) ** i, math.factorial(2 * i)))
                                           for i in range(1, 7)]
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120

    def near_mp(x):
        return nearest32(Fraction(int(mpmath.nint(x * mpmath.mpf(2) ** 110)), 2 ** 110))

    assert float(ph._LN2) == near_mp(mpmath.log(2))
    assert float(ph._HALF_PI) == near_mp(mpmath.pi / 2)
    assert float(ph._SQRT_HALF) == near_mp(mpmath.sqrt(mpmath.mpf(1) / 2))


def test_ln_series_against_libm():
    # binary32 series against binary64 libm: within 3 binary32 ulps
    g = np.random.default_rng(11)
    u = ph.uniform_from_u64(g.integers(0, 2**63, size=400000, dtype=np.int64).astype(np.uint64) * np.uint64(2))
    edge = np.float32([2.0**-24, 2.0**-23 * 1.5, 0.5, 0.70710677, 0.70710683, 0.99999994])
    u = np.concatenate([u, edge])
    got = ph.ln_series(u)
    assert got.dtype == np.float32
    ref = np.log(u.astype(np.float64))
    ulp = np.abs(got.astype(np.float64) - ref) / np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert ulp.max() <= 3.0


def test_sincos_against_mpmath():
    # binary32 series against 120-bit sin / cos: within 2^-23 absolute
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    g = np.random.default_rng(12)
    u = np.concatenate([g.random(1500).astype(np.float32),
                        np.float32([0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 2.0**-23, 1 - 2.0**-24])])
    s, c = ph.sincos_2pi(u)
    assert s.dtype == np.float32 and c.dtype == np.float32
    rs = np.array([float(mpmath.sin(2 * mpmath.pi * mpmath.mpf(float(x)))) for x in u])
    rc = np.array([float(mpmath.cos(2 * mpmath.pi * mpmath.mpf(float(x)))) for x in u])
    assert np.abs(s - rs).max() <= 2.0**-23
    assert np.abs(c - rc).max() <= 2.0**-23


def test_gaussian_moments_and_ks():
    om = ph.gaussian_matrix(2000, 600, seed=3)
    z = om.ravel()
    N = z.size
    assert abs(z.mean()) < 5 / np.sqrt(N)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / N)
    assert abs(stats.skew(z)) < 5 * np.sqrt(6 / N)
    assert abs(stats.kurtosis(z)) < 5 * np.sqrt(24 / N)
    assert stats.kstest(z[:200000], "norm").pvalue > 1e-4


def test_column_major_element_order_and_streams():
    n, l = 37, 5
    om = ph.gaussian_matrix(n, l, seed=9)
    i, j = np.meshgrid(np.arange(n), np.arange(l), indexing="ij")
    e = (i + n * j).ravel()
    assert np.array_equal(om.ravel(), ph.gaussian_elements(e, 9))
    other = ph.gaussian_matrix(n, l, seed=9, stream=1)
    assert not np.any(other == om)
    assert not np.any(ph.gaussian_matrix(n, l, seed=10) == om)


def test_reduced_precision_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = ph.gaussian_matrix(64, 64, seed=1).ravel()
    f32 = torch.tensor(x, dtype=torch.float64).to(torch.float32)
    assert np.array_equal(ph.round_to(x, "f32"), f32.double().numpy())
    assert np.array_equal(ph.round_to(x, "bf16"), f32.to(torch.bfloat16).double().numpy())
    assert np.array_equal(ph.round_to(x, "f16"), f32.to(torch.float16).double().numpy())

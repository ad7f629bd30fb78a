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
    x = np.array([0, 1, 2**12 - 1, 2**12, 2**63, 2**64 - 1], dtype=np.uint64)
    u = ph.uniform_from_u64(x)
    assert np.all(u > 0) and np.all(u < 1)
    k = u * 2.0**52 - 0.5
    assert np.array_equal(k, np.floor(k))
    assert np.array_equal(k.astype(np.uint64), x >> np.uint64(12))


def test_ln_series_against_libm():
    g = np.random.default_rng(11)
    u = ph.uniform_from_u64(g.integers(0, 2**63, size=400000, dtype=np.int64).astype(np.uint64) * np.uint64(2))
    edge = np.array([2.0**-53, 2.0**-52 * 1.5, 0.5, 0.70710678118654746, 0.70710678118654757,
                     0.99999999999999989, 1.0 - 2.0**-52])
    u = np.concatenate([u, edge])
    got = ph.ln_series(u)
    ref = np.log(u)
    ulp = np.abs(got - ref) / np.spacing(np.abs(ref))
    assert ulp.max() <= 4.0


def test_sincos_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    g = np.random.default_rng(12)
    u = np.concatenate([g.random(1500), [0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875, 2.0**-52, 1 - 2.0**-52]])
    s, c = ph.sincos_2pi(u)
    rs = np.array([float(mpmath.sin(2 * mpmath.pi * mpmath.mpf(float(x)))) for x in u])
    rc = np.array([float(mpmath.cos(2 * mpmath.pi * mpmath.mpf(float(x)))) for x in u])
    assert np.abs(s - rs).max() <= 2.3e-16
    assert np.abs(c - rc).max() <= 2.3e-16


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

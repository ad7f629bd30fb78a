"""The library's bound evaluator (sorsvd_bounds: Theorems 4-7 of Sec. IV,
host code) against the oracle's bounds module - two independent
restatements of the same formulas - on synthetic spectra with known right
singular vectors and Gaussian test matrices, and at the hand-computed values
that pin the oracle; plus its argument checks.  No GPU."""
import math

import numpy as np
import pytest

from oracle import bounds as ob
from oracle.philox import gaussian_matrix


@pytest.fixture(scope="module")
def nat():
    from paper_1804_00462_gb300 import native
    return native


def _norms(V, omega, k):
    O1 = V[:, :k].T @ omega
    O2 = V[:, k:].T @ omega
    return float(np.linalg.norm(O2, 2)), float(1.0 / np.linalg.svd(O1, compute_uv=False)[-1])


@pytest.mark.parametrize("n,k,p,q,decay", [(60, 5, 3, 0, "poly"), (80, 10, 5, 1, "exp"), (120, 20, 8, 2, "poly"),
                                           (50, 3, 0, 1, "exp")])
def test_matches_the_oracle_bounds(nat, n, k, p, q, decay):
    j = np.arange(1, n + 1, dtype=np.float64)
    sigma = 1.0 / j if decay == "poly" else np.exp(-j / 8.0)
    V, _ = np.linalg.qr(np.random.default_rng(n).standard_normal((n, n)))
    omega = gaussian_matrix(n, k + p, seed=k, stream=0, dtype="f64")
    o2, o1 = _norms(V, omega, k)
    got = nat.bounds(sigma, n, k, p, q, o2, o1)
    assert np.allclose(got["thm4_lower"], ob.thm4_lower(sigma, V, omega, k, q), rtol=1e-12, atol=0)
    assert math.isclose(got["thm5_upper_2"], ob.thm5_upper(sigma, V, omega, k, q, "2"), rel_tol=1e-12)
    assert math.isclose(got["thm5_upper_fro"], ob.thm5_upper(sigma, V, omega, k, q, "fro"), rel_tol=1e-12)
    assert np.allclose(got["thm6_lower"], ob.thm6_expected_lower(sigma, n, k, p, q), rtol=1e-12, atol=0)
    assert math.isclose(got["thm7_upper_2"], ob.thm7_expected_upper(sigma, n, k, p, q, "2"), rel_tol=1e-12)
    assert math.isclose(got["thm7_upper_fro"], ob.thm7_expected_upper(sigma, n, k, p, q, "fro"), rel_tol=1e-12)
    assert got["ey_2"] == sigma[k] and math.isclose(got["ey_fro"], math.sqrt(np.sum(sigma[k:] ** 2)), rel_tol=1e-13)


def test_hand_computed_values(nat):
    # A = diag(2, 1, 1/2, 1/4), k = 1, p = 2, x = (||Omega2|| ||Omega1^+||)^2 = 1/4
    # (||Omega2||_2 = 1, ||Omega1^+||_2 = 1/2); the values are worked out in
    # the oracle's pin of the same case
    s = [2.0, 1.0, 0.5, 0.25]
    r3, r17, r65, r257, r1025 = (math.sqrt(v) for v in (3.0, 17.0, 65.0, 257.0, 1025.0))
    a0f = math.sqrt(21.0) / 4
    nu = (7 + 2 * r3) * 4 * math.e * r3 / 3
    b0 = nat.bounds(s, 4, 1, 2, 0, 1.0, 0.5)
    b1 = nat.bounds(s, 4, 1, 2, 1, 1.0, 0.5)
    assert math.isclose(b0["thm4_lower"][0], 16 / r65, rel_tol=1e-14)
    assert math.isclose(b1["thm4_lower"][0], 64 / r1025, rel_tol=1e-14)
    assert math.isclose(b0["thm5_upper_2"], 1 + 2 / r65 + 2 / r17, rel_tol=1e-14)
    assert math.isclose(b0["thm5_upper_fro"], a0f + 2 / r65 + 2 / r17, rel_tol=1e-14)
    assert math.isclose(b1["thm5_upper_2"], 1 + 2 / r1025 + 2 / r257, rel_tol=1e-14)
    assert math.isclose(b0["thm6_lower"][0], 2 / math.sqrt(1 + nu ** 2 / 16), rel_tol=1e-14)
    assert math.isclose(b1["thm6_lower"][0], 2 / math.sqrt(1 + nu ** 2 / 256), rel_tol=1e-14)
    assert math.isclose(b0["thm7_upper_2"], 1 + 1.5 * nu, rel_tol=1e-14)
    assert math.isclose(b1["thm7_upper_fro"], a0f + 0.375 * nu, rel_tol=1e-14)


def test_exact_rank_and_unknown_omega(nat):
    # sigma_{k+1} = 0: every bound collapses onto the exact value
    b = nat.bounds([3.0, 2.0, 1.0, 0.0, 0.0], 10, 3, 2, 1, 1.5, 2.0)
    assert b["ey_2"] == 0.0 and b["thm5_upper_2"] == 0.0 and b["thm7_upper_fro"] == 0.0
    assert b["thm4_lower"] == [3.0, 2.0, 1.0] and b["thm6_lower"] == [3.0, 2.0, 1.0]
    u = nat.bounds([3.0, 2.0, 1.0, 0.5], 10, 2, 2, 0)
    assert math.isnan(u["thm5_upper_2"]) and all(math.isnan(v) for v in u["thm4_lower"])
    assert math.isfinite(u["thm7_upper_2"])


def test_argument_checks(nat):
    from paper_1804_00462_gb300.native import SorsvdError
    for args in [([1.0, 2.0, 0.5], 10, 1, 1, 0),      # increasing sigma
                 ([1.0, 0.5], 10, 2, 1, 0),           # r < k + 1
                 ([1.0, 0.0, 0.0], 10, 2, 1, 0),      # sigma_k = 0
                 ([1.0, 0.5, 0.2], 2, 2, 1, 0),       # n < k + p
                 ([1.0, -0.5, 0.2], 10, 1, 1, 0)]:    # negative
        with pytest.raises(SorsvdError):
            nat.bounds(*args)

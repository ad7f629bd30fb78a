"""Pins of the oracle's inexact-ALM RPCA with SOR-SVD inside (Table 3):
the soft-threshold operator's closed form and the recovery behaviour the
paper reports for synthetic data (Sec. V-C-1, Tables 4-5: the rank of L and
the support of S are recovered exactly, relative error below 1e-7 after a
few tens of iterations)."""
import numpy as np

from oracle.rpca import rpca_alm, shrink
from paper_1804_00462_gb300 import inputs


def test_shrink_closed_form():
    x = np.array([-3.0, -1.0, -0.5, 0.0, 0.2, 1.0, 4.0])
    assert np.array_equal(shrink(x, 1.0), np.array([-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 3.0]))
    # shrink is the proximal map of eps*|.|: argmin_y 0.5 (y - x)^2 + eps |y|
    g = np.random.default_rng(0)
    x = g.standard_normal(200) * 3
    ys = np.linspace(-12, 12, 240001)
    for xi in x[:20]:
        best = ys[np.argmin(0.5 * (ys - xi) ** 2 + 0.7 * np.abs(ys))]
        assert abs(best - shrink(np.array([xi]), 0.7)[0]) <= 1e-4


def test_rpca_recovers_rank_and_support():
    X, L0, S0 = inputs.rpca_problem(m=1200, n=200, rank=5, density=0.05, seed=1)
    out = rpca_alm(X, 5, 5, 1, seed=0, norm2=float(np.linalg.norm(X, 2)))
    assert out["xi"] < 1e-7
    assert out["iters"] <= 50
    sv = np.linalg.svd(out["L"], compute_uv=False)
    assert np.sum(sv > 1e-6 * sv[0]) == 5
    assert np.array_equal(np.abs(out["S"]) > 1e-3, S0 != 0)
    assert np.linalg.norm(out["L"] - L0) <= 1e-5 * np.linalg.norm(L0)

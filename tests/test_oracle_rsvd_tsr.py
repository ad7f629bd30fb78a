"""Pins of the oracle's comparison methods (Sec. II): the randomized SVD
R-SVD (Algorithm 1) and the two-sided randomized SVD TSR-SVD (Algorithm 2).

- Exact recovery: for rank(A) = r <= l both reproduce A (R-SVD: range(Q) is
  range(A); TSR-SVD: range(Q2) is the row space of A, so A Psi1 =
  A Q2 Q2^T Psi1 and B_approx = Q1^T A Q2 exactly).
- R-SVD equals SOR-SVD with the same Omega and q: Q is SOR-SVD's Q1, and
  the rows of B = Q^T A lie in range(Q2) (Q2 spans A^T Q1), so
  [B]_k = [Q1^T A Q2]_k Q2^T and the rank-k approximations coincide.
- R-SVD's singular values are those of B = Q^T A (a LAPACK SVD of the same
  l x n matrix), and Eckart-Young bounds every rank-k error from below.
- A planted mistake (the columns of B mixed up before its SVD) is caught."""
import numpy as np
import pytest

from oracle import sor_svd as orc
from oracle.linalg import householder_qr
from oracle.philox import gaussian_matrix
from paper_1804_00462_gb300 import inputs


def _rel(A, U, S, V):
    return orc.recon_error_fro(A, U, S, V) / np.linalg.norm(A)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rsvd_exact_recovery(q):
    A = inputs.exact_rank(260, 180, 10, seed=q + 5)
    U, S, V = orc.rsvd(A, 10, 4, q, seed=3)
    assert _rel(A, U, S, V) < 1e-12
    assert np.linalg.norm(U.T @ U - np.eye(10)) < 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(10)) < 1e-12


def test_tsrsvd_exact_recovery():
    for (m, n, r, k, p, seed) in [(200, 150, 8, 8, 4, 1), (90, 240, 5, 7, 3, 2)]:
        A = inputs.exact_rank(m, n, r, seed=seed)
        U, S, V = orc.tsrsvd(A, k, p, seed=seed)
        assert _rel(A, U, S, V) < 1e-11, (m, n, r)
        assert np.all(S[r:] < 1e-11 * S[0])


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("mode", ["stabilised", "literal"])
def test_rsvd_equals_sorsvd_for_the_same_omega(q, mode):
    A = inputs.spectral(220, 160, inputs.sigma_poly(160, 1.0), seed=7)[0]
    k, p = 12, 6
    Ur, Sr, Vr = orc.rsvd(A, k, p, q, seed=9, mode=mode)
    Us, Ss, Vs = orc.sorsvd(A, k, p, q, seed=9, mode=mode)
    Ar = (Ur * Sr) @ Vr.T
    As = (Us * Ss) @ Vs.T
    assert np.linalg.norm(Ar - As) <= 1e-10 * np.linalg.norm(A)
    assert np.allclose(Sr, Ss, rtol=1e-10, atol=0)


def test_rsvd_singular_values_are_those_of_b():
    A = inputs.spectral(150, 120, inputs.sigma_poly(120, 2.0), seed=2)[0]
    k, p, q = 10, 5, 1
    U, S, V = orc.rsvd(A, k, p, q, seed=4)
    Y = A @ gaussian_matrix(120, k + p, 4, 0, "f64")
    Y = A @ (A.T @ householder_qr(Y)[0])
    Q = householder_qr(Y)[0]
    s_ref = np.linalg.svd(Q.T @ A, compute_uv=False)
    assert np.allclose(S, s_ref[:k], rtol=1e-12, atol=0)


@pytest.mark.parametrize("method", ["rsvd", "tsrsvd"])
def test_eckart_young_lower_bound(method):
    sig = inputs.sigma_poly(100, 1.0)
    A = inputs.spectral(140, 100, sig, seed=3)[0]
    k, p = 10, 5
    U, S, V = orc.rsvd(A, k, p, 0, seed=1) if method == "rsvd" else orc.tsrsvd(A, k, p, seed=1)
    _, ey = orc.eckart_young(sig, k)
    assert orc.recon_error_fro(A, U, S, V) >= ey * (1 - 1e-12)


def test_planted_scrambled_b_is_caught(monkeypatch):
    # the rows of B^T (columns of B) permuted before the SVD: exact recovery fails
    A = inputs.exact_rank(120, 80, 6, seed=11)
    U, S, V = orc.rsvd(A, 6, 4, 0, seed=2)
    assert _rel(A, U, S, V) < 1e-12
    real_svd = orc.jacobi_svd

    def wrong(M, *a, **kw):
        return real_svd(M[::-1].copy(), *a, **kw)
    monkeypatch.setattr(orc, "jacobi_svd", wrong)
    U2, S2, V2 = orc.rsvd(A, 6, 4, 0, seed=2)
    assert _rel(A, U2, S2, V2) > 1e-3

"""Pins of the oracle's Householder QR and one-sided Jacobi SVD against LAPACK
(numpy / scipy) and the defining properties of each factorisation."""
import itertools

import numpy as np
import pytest

from oracle.linalg import EPS64, _tournament_rounds, householder_qr, jacobi_svd


@pytest.mark.parametrize("n", [1, 2, 5, 8, 25, 33])
def test_tournament_covers_every_pair_once(n):
    seen = []
    for pairs in _tournament_rounds(n):
        flat = [x for pq in pairs for x in pq]
        assert len(flat) == len(set(flat))          # disjoint within a round
        seen += pairs
    assert sorted(seen) == sorted(itertools.combinations(range(n), 2))


@pytest.mark.parametrize("m,l", [(50, 7), (300, 40), (64, 64), (1000, 25)])
def test_householder_qr_against_lapack(m, l):
    T = np.random.default_rng(m * 7 + l).standard_normal((m, l))
    Q, R = householder_qr(T)
    assert np.allclose(np.triu(R), R)
    assert np.all(np.diag(R) >= 0)
    assert np.linalg.norm(Q @ R - T) <= 50 * EPS64 * np.linalg.norm(T)
    assert np.linalg.norm(Q.T @ Q - np.eye(l)) <= 10 * l * EPS64
    Ql, Rl = np.linalg.qr(T)
    d = np.sign(np.diag(Rl))
    assert np.allclose(Q, Ql * d, atol=1e-12)
    assert np.allclose(R, Rl * d[:, None], atol=1e-12 * np.abs(Rl).max())


def test_householder_qr_rank_deficient_stays_orthonormal():
    g = np.random.default_rng(5)
    T = g.standard_normal((200, 4)) @ g.standard_normal((4, 12))
    T[:, 7] = 0.0
    Q, R = householder_qr(T)
    assert np.linalg.norm(Q.T @ Q - np.eye(12)) <= 1e-13
    assert np.linalg.norm(Q @ R - T) <= 1e-13 * np.linalg.norm(T)


@pytest.mark.parametrize("r,c", [(6, 6), (40, 40), (110, 110), (90, 31)])
def test_jacobi_svd_against_lapack(r, c):
    g = np.random.default_rng(r + 1000 * c)
    M = g.standard_normal((r, c)) * np.logspace(0, -6, c)[None, :]
    U, s, V, sweeps = jacobi_svd(M)
    ref = np.linalg.svd(M, compute_uv=False)
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s - ref)) <= 1e-13 * ref[0]
    assert np.linalg.norm((U * s) @ V.T - M) <= 1e-13 * np.linalg.norm(M)
    assert np.linalg.norm(U.T @ U - np.eye(c)) <= 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(c)) <= 1e-12
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(c)] > 0)
    assert sweeps < 30


def test_jacobi_svd_singular_input():
    g = np.random.default_rng(3)
    M = g.standard_normal((20, 3)) @ g.standard_normal((3, 20))
    U, s, V, _ = jacobi_svd(M)
    ref = np.linalg.svd(M, compute_uv=False)
    assert np.max(np.abs(s - ref)) <= 1e-13 * ref[0]
    assert np.linalg.norm((U * s) @ V.T - M) <= 1e-13 * np.linalg.norm(M)
    assert np.all(s[3:] <= 1e-13 * s[0])


def test_jacobi_svd_diagonal_and_permuted():
    d = np.array([3.0, -1.0, 7.0, 0.5])
    U, s, V, _ = jacobi_svd(np.diag(d))
    assert np.array_equal(s, np.array([7.0, 3.0, 1.0, 0.5]))
    assert np.allclose(np.abs(U), np.abs(V))
